// Host-side launch interface between the C-ABI layer and the kernels.
#pragma once

#include "ens_internal.h"

namespace ens {

enum class Pass { IX, IY, Z, FY, FX, ZSTAT };
// IY mode of the statistics snapshot: the eight gradient components from the
// six x-pass fields (u_i, i kx u_i)
constexpr int kIYGrad = -1;

// lambda-weight specification on the device (kind: 0 Gaussian with the
// paper's mean and variance from c and Z, 1 Gaussian (mu, sigma), 2 user
// weights, 3 truncated Gaussian from c and Z)
struct MixWeightArgs {
    int kind;
    double c, Z, mu, sigma;
    const double *user;
    int renormalize;
};

struct MixPdfArgs {
    int nq, nt, ng, counts_len;
    double dq, dr, dt, dg;   // bin widths: Q/q0, R/q0^1.5, log10 tail axis, A/sqrt(q0)
};
// mixed PDF values: [nq*nq | nt | nt | ng (longitudinal) | ng (transverse)]
__host__ __device__ inline int mix_pdf_len(const MixPdfArgs &a) { return a.nq * a.nq + 2 * a.nt + 2 * a.ng; }

bool supported_n(int N);
int plan_threads(int N);
int stats_blocks(int N);
size_t stats_smem(int N, int nq, int nt, int ng);   // shared memory per CTA of the statistics pass
cudaError_t prepare_kernels(int N, int nq, int nt, int ng);
int znl_ctas_per_sm(int N, int var = 0);   // resident CTAs per SM of the persistent z pass (0 on error)
bool zplan_variant_available(int N);       // the persistent z pass has a second warp plan for this size
bool plan_variant_available(int N);   // the x passes have a second FFT plan for this size
bool fx_ws_available(int N);          // the last pass has its warp-group variant (fx_split 2) for this size

// Pass launchers of one grid size (ens_sized.cu, one translation unit per N).
struct SizedOps {
    cudaError_t (*prepare)(int nq, int nt, int ng);
    int (*znl_ctas_per_sm)(int var);
    void (*launch)(Pass pass, int mode, const Geo &g, MemberDev *md, const HistDev *h, int stage, int last,
                   int arg, cudaStream_t s);
    bool (*fx_ws)();   // the warp-group variant of the last pass exists for this size
};
template <int N>
const SizedOps *sized_ops_for();
#define ENS_DECLARE_SIZED(n) template <> const SizedOps *sized_ops_for<n>();
ENS_DECLARE_SIZED(16)
ENS_DECLARE_SIZED(32)
ENS_DECLARE_SIZED(64)
ENS_DECLARE_SIZED(128)
ENS_DECLARE_SIZED(256)
ENS_DECLARE_SIZED(384)
ENS_DECLARE_SIZED(512)
#undef ENS_DECLARE_SIZED
const SizedOps *sized_ops(int N);   // nullptr for an unsupported size

// mode/arg per pass:
//   IX: mode 0 (u, omega) or 1 (gradient), arg = read S instead of U
//   IY: mode = first field, arg = number of fields
//   Z : mode 0 nonlinear, 1 noise, 3 velocity to physical, 4 physical to spectral
//   FY: forward along y of fields 0..2
//   FX: mode 0 RK update, 1 right-hand side, 2 initial field, 3 plain transform
//   ZSTAT: statistics
// The stage passes (IX mode 0, IY, FY, FX mode 0, Z mode 0) take their
// variant from the group's tuning in g (tile_x, tile_y, plan_x, fx_split,
// z_mode: 0 persistent, 1 row groups, 2 persistent with the second warp plan).
void launch_pass(Pass pass, int mode, const Geo &g, MemberDev *md, const HistDev *h, int stage, int last, int arg,
                 cudaStream_t s);
void launch_state_sums(const Geo &g, MemberDev *md, cudaStream_t s);
void launch_finish(MemberDev *md, int nmembers, const double *partial, int partial_blocks, int stage, int last,
                   int mode, cudaStream_t s);
void launch_ic(const Geo &g, MemberDev *md, cudaStream_t s);
void launch_twiddles(float2 *tw, int N, cudaStream_t s);
void launch_edges(float *eq, float *er, float *et, float *eg, int nq, int nt, int ng, double q_lim, double r_lim,
                  double t_lo, double t_hi, double g_lim, cudaStream_t s);
void launch_finish_stats(const double *mom_partial, int blocks, double *moments, int nmembers, int accumulate,
                         cudaStream_t s);
void launch_bin_check(const HistDev &h, int axis, const float *x, int n, int *out, cudaStream_t s);
void launch_mixture(const double *lam, int n, const MixWeightArgs &wa, const unsigned long long *counts,
                    const double *moments, const MixPdfArgs &pa, double *w, double *covered, double *pdf,
                    double *mom_mix, double *ratios, cudaStream_t s);

}  // namespace ens
