// Host-side launch interface between the C-ABI layer and the kernels.
#pragma once

#include "ens_internal.h"

namespace ens {

enum class Pass { IX, IY, Z, FY, FX, ZSTAT };

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
    int nq, nt, counts_len;
    double dq, dr, dt;   // bin widths: Q/q0, R/q0^1.5, log10 tail axis
};

bool supported_n(int N);
int plan_threads(int N);
int stats_blocks(int N);
cudaError_t prepare_kernels(int N, int nq, int nt);
int znl_ctas(int N);   // persistent grid of the z nonlinear pass (0 on error)

// mode/arg per pass:
//   IX: mode 0 (u, omega) or 1 (gradient), arg = read S instead of U
//   IY: mode = first field, arg = number of fields
//   Z : mode 0 nonlinear, 1 noise, 3 velocity to physical, 4 physical to spectral
//   FY: forward along y of fields 0..2
//   FX: mode 0 RK update, 1 right-hand side, 2 initial field, 3 plain transform
//   ZSTAT: statistics
void launch_pass(Pass pass, int mode, const Geo &g, MemberDev *md, const HistDev *h, int stage, int last, int arg,
                 cudaStream_t s);
void launch_state_sums(const Geo &g, MemberDev *md, cudaStream_t s);
void launch_finish(MemberDev *md, int nmembers, const double *partial, int partial_blocks, int stage, int last,
                   int mode, cudaStream_t s);
void launch_ic(const Geo &g, MemberDev *md, cudaStream_t s);
void launch_twiddles(float2 *tw, int N, cudaStream_t s);
void launch_edges(float *eq, float *er, float *et, int nq, int nt, double q_lim, double r_lim, double t_lo,
                  double t_hi, cudaStream_t s);
void launch_finish_stats(const double *mom_partial, int blocks, double *moments, int nmembers, int accumulate,
                         cudaStream_t s);
void launch_mixture(const double *lam, int n, const MixWeightArgs &wa, const unsigned long long *counts,
                    const double *moments, const MixPdfArgs &pa, double *w, double *covered, double *pdf,
                    double *mom_mix, double *ratios, cudaStream_t s);

}  // namespace ens
