// Non-templated kernels (reductions, initial field, twiddles, edges, mixture)
// and the table of per-N pass launchers (each grid size compiles in its own
// translation unit, ens_sized.cu).
#include "ens_launch.h"
#include "ens_stats.cuh"
#include "ens_znl.cuh"

#include <cmath>

namespace ens {

// ---------------------------------------------------------------------------
// spectral sums of U (init / after upload), same partial layout as FXU
// ---------------------------------------------------------------------------
__global__ void k_state_sums(Geo g, MemberDev *md)
{
    const int m = blockIdx.y;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;   // (ky, kz) flat
    const int ncols = g.NK * g.NZp;
    const MemberDev &d = md[g.first + m];
    float se = 0.f, sd = 0.f, sb = 0.f;
    if (col < ncols) {
        const int iy = col / g.NZp, kz = col % g.NZp;
        if (kz < g.NZ) {
            const int ky = iy <= g.kc ? iy : iy - g.NK;
            const float wgt = kz == 0 ? 1.f : 2.f;
            const float2 *U = g.U + (long long)m * 3 * g.sU + col;
            for (int ix = 0; ix < g.NK; ++ix) {
                const int kx = ix <= g.kc ? ix : ix - g.NK;
                const int k2i = kx * kx + ky * ky + kz * kz;
                float a2 = 0.f;
                for (int q = 0; q < 3; ++q) {
                    const float2 v = U[q * g.sU + (long long)ix * ncols];
                    a2 += v.x * v.x + v.y * v.y;
                }
                se += 0.5f * wgt * a2;
                sd += (float)d.nu * (float)k2i * wgt * a2;
                if (k2i >= d.band_lo2 && k2i <= d.band_hi2) sb += 0.5f * wgt * a2;
            }
        }
    }
    __shared__ double scratch[32 * 3];
    double vals[3] = {(double)se, (double)sd, (double)sb};
    double *out = g.partial + ((long long)(g.first + m) * g.partial_blocks + blockIdx.x) * 4;
    block_sum_to<3>(out, vals, scratch);
}

__global__ void k_finish(MemberDev *md, const double *partial, int partial_blocks, int stage, int last_stage,
                         int mode)
{
    finish_body(md, partial, partial_blocks, stage, last_stage, mode, blockIdx.x, threadIdx.x);
}

// ---------------------------------------------------------------------------
// initial field: shell targets E0(s) ~ s^4 exp(-s^2/2), total init_energy
// ---------------------------------------------------------------------------
__global__ void k_ic_factors(MemberDev *md, Geo g)
{
    const int m = blockIdx.x;
    double *shell = g.shell + (long long)m * g.shells;
    __shared__ double total;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int s = 1; s < g.shells; ++s)
            if (shell[s] > 0.0) t += pow((double)s, 4.0) * exp(-0.5 * s * s);
        total = t;
    }
    __syncthreads();
    const double E0 = md[g.first + m].init_energy;
    for (int s = threadIdx.x; s < g.shells; s += blockDim.x) {
        double f = 0.0;
        if (s > 0 && shell[s] > 0.0 && total > 0.0)
            f = sqrt(E0 * pow((double)s, 4.0) * exp(-0.5 * s * s) / (total * shell[s]));
        shell[s] = f;   // shell sums are replaced by the rescaling factors
    }
}

__global__ void k_ic_scale(Geo g)
{
    const int m = blockIdx.y;
    const long long ncols = (long long)g.NK * g.NZp;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // (kx, ky, kz) flat
    if (idx >= (long long)g.NK * ncols) return;
    const int ix = (int)(idx / ncols);
    const int col = (int)(idx % ncols);
    const int iy = col / g.NZp, kz = col % g.NZp;
    float2 *U = g.U + (long long)m * 3 * g.sU + idx;
    if (kz >= g.NZ) {
        for (int q = 0; q < 3; ++q) U[q * g.sU] = make_float2(0.f, 0.f);
        return;
    }
    const int kx = ix <= g.kc ? ix : ix - g.NK, ky = iy <= g.kc ? iy : iy - g.NK;
    const int s = (int)lrint(sqrt((double)(kx * kx + ky * ky + kz * kz)));
    const float f = (float)g.shell[(long long)m * g.shells + s];
    for (int q = 0; q < 3; ++q) U[q * g.sU] = cscale(U[q * g.sU], f);
}

__global__ void k_twiddles(float2 *tw, int N)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)i / (double)N, &s, &c);
        tw[i] = make_float2((float)c, (float)s);
    }
}

__global__ void k_edges(float *eq, float *er, float *et, float *eg, int nq, int nt, int ng, double q_lim,
                        double r_lim, double t_lo, double t_hi, double g_lim)
{
    for (int b = threadIdx.x; b <= ng; b += blockDim.x) eg[b] = (float)(-g_lim + 2.0 * g_lim * (double)b / (double)ng);
    for (int b = threadIdx.x; b <= nq; b += blockDim.x) {
        eq[b] = (float)(-q_lim + 2.0 * q_lim * (double)b / (double)nq);
        er[b] = (float)(-r_lim + 2.0 * r_lim * (double)b / (double)nq);
    }
    for (int b = threadIdx.x; b <= nt; b += blockDim.x)
        et[b] = (float)pow(10.0, t_lo + (t_hi - t_lo) * (double)b / (double)nt);
}

__global__ void k_finish_stats(const double *mom_partial, int blocks, double *moments, int accumulate)
{
    const int gm = blockIdx.x, t = threadIdx.x;
    if (t >= kNMom) return;
    double s = 0.0;
    const double *pp = mom_partial + (long long)gm * blocks * kNMom;
    for (int b = 0; b < blocks; ++b) s += pp[(long long)b * kNMom + t];
    moments[gm * kNMom + t] = accumulate ? moments[gm * kNMom + t] + s : s;
}

// ---------------------------------------------------------------------------
// mixture (Sec. II, Eqs. ensemble_hypothesis / pdf_superposition; Sec. IV,
// Eq. gaussian_lambda_pdf and the lambda-bin weights; Appendix,
// Eq. truncated_gaussian), FP64
// ---------------------------------------------------------------------------
__device__ double norm_cdf(double x) { return 0.5 * erfc(-x * 0.70710678118654752440); }
__device__ double norm_sf(double x) { return 0.5 * erfc(x * 0.70710678118654752440); }

__device__ double interval_mass(double a, double b, double mu, double sigma)
{
    const double za = (a - mu) / sigma, zb = (b - mu) / sigma;
    if (za >= 0.0) return norm_sf(za) - norm_sf(zb);
    return norm_cdf(zb) - norm_cdf(za);
}

// mu of the truncated Gaussian so that int P e^lambda = 1 (bisection in logs)
__device__ double trunc_mu(double c, double Z)
{
    const double sigma = sqrt(9.0 * c * Z);
    double lo = -4.5 * c * Z - 10.0 * sigma - 1.0, hi = 10.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        const double f = mid + 0.5 * sigma * sigma + log(norm_cdf((Z - mid - sigma * sigma) / sigma)) -
                         log(norm_cdf((Z - mid) / sigma));
        if (f < 0.0) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

__global__ void k_mix_weights(const double *lam, int n, MixWeightArgs wa, double *w, double *covered)
{
    const int i = threadIdx.x;
    __shared__ double wsh[1024];
    if (i < n) {
        const double li = lam[i];
        double prev = -INFINITY, next = INFINITY;
        int mult = 0;
        for (int j = 0; j < n; ++j) {
            const double lj = lam[j];
            if (lj == li) ++mult;
            else if (lj < li && lj > prev) prev = lj;
            else if (lj > li && lj < next) next = lj;
        }
        double lo, hi;
        if (prev == -INFINITY && next == INFINITY) {
            lo = -INFINITY;
            hi = INFINITY;
        } else {
            lo = prev == -INFINITY ? li - 0.5 * (next - li) : 0.5 * (prev + li);
            hi = next == INFINITY ? li + 0.5 * (li - prev) : 0.5 * (li + next);
        }
        double v = 0.0;
        if (wa.kind == 2) {
            v = wa.user[i];
        } else if (wa.kind == 0 && wa.Z == 0.0) {
            v = (lo <= 0.0 && 0.0 < hi) ? 1.0 / mult : 0.0;
        } else if (wa.kind == 0 || wa.kind == 1) {
            const double mu = wa.kind == 0 ? -4.5 * wa.c * wa.Z : wa.mu;
            const double sg = wa.kind == 0 ? sqrt(9.0 * wa.c * wa.Z) : wa.sigma;
            v = interval_mass(lo, hi, mu, sg) / mult;
        } else if (wa.kind == 3) {
            const double mu = trunc_mu(wa.c, wa.Z), sg = sqrt(9.0 * wa.c * wa.Z);
            const double b = fmin(hi, wa.Z);
            v = b > lo ? interval_mass(lo, b, mu, sg) / norm_cdf((wa.Z - mu) / sg) / mult : 0.0;
        }
        wsh[i] = v;
    }
    __syncthreads();
    __shared__ double tot;
    if (i == 0) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += wsh[j];
        tot = s;
        *covered = s;
    }
    __syncthreads();
    if (i < n) w[i] = (wa.renormalize && tot > 0.0) ? wsh[i] / tot : wsh[i];
}

__global__ void k_mix_pdf(const unsigned long long *counts, const double *moments, const double *w, int n,
                          MixPdfArgs a, double *pdf, double *mom_mix)
{
    const int L = a.counts_len;
    const int off_c = a.nq * a.nq + 2 * a.nt;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < mix_pdf_len(a)) {
        // gradient bins follow the 8 counters; 3 longitudinal and 6
        // transverse samples per grid point
        const bool grad = b >= off_c;
        const int src = grad ? b + 8 : b;
        double s = 0.0;
        for (int i = 0; i < n; ++i) {
            const double npts = (double)counts[(long long)i * L + off_c + 6];
            if (npts > 0.0) s += w[i] * (double)counts[(long long)i * L + src] / npts;
        }
        double width = b < a.nq * a.nq ? a.dq * a.dr : a.dt;
        if (grad) width = a.dg * (b < off_c + a.ng ? 3.0 : 6.0);
        pdf[b] = s / width;
    }
    if (blockIdx.x == 0 && threadIdx.x < kNMom) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) {
            const double npts = (double)counts[(long long)i * L + off_c + 6];
            if (npts > 0.0) s += w[i] * moments[(long long)i * kNMom + threadIdx.x] / npts;
        }
        mom_mix[threadIdx.x] = s;
    }
}

// skewness / flatness / hyper-flatness of gradient components from mixed
// moments (Sec. VII, Eq. def_skewness_flatness and the skewness prediction),
// isotropy-averaged over the 3 longitudinal and 6 transverse components
__global__ void k_mix_ratios(const double *mom_mix, double *ratios)
{
    if (threadIdx.x != 0) return;
    const int lon[3] = {0, 4, 8}, tra[6] = {1, 2, 3, 5, 6, 7};
    double L[4] = {0, 0, 0, 0}, T[4] = {0, 0, 0, 0};
    for (int q = 0; q < 4; ++q) {
        for (int c = 0; c < 3; ++c) L[q] += mom_mix[4 * lon[c] + q] / 3.0;
        for (int c = 0; c < 6; ++c) T[q] += mom_mix[4 * tra[c] + q] / 6.0;
    }
    ratios[0] = L[1] / pow(L[0], 1.5);
    ratios[1] = L[2] / (L[0] * L[0]);
    ratios[2] = T[2] / (T[0] * T[0]);
    ratios[3] = L[3] / (L[0] * L[0] * L[0]);
    ratios[4] = T[3] / (T[0] * T[0] * T[0]);
}

// ---------------------------------------------------------------------------
// launch dispatch
// ---------------------------------------------------------------------------
#define ENS_SUPPORTED_N(X) X(16) X(32) X(64) X(128) X(256) X(384) X(512)

bool supported_n(int N)
{
#define X(n) if (N == n) return true;
    ENS_SUPPORTED_N(X)
#undef X
    return false;
}

int plan_threads(int N)
{
#define X(n) if (N == n) return PlanInfo<n>::P;
    ENS_SUPPORTED_N(X)
#undef X
    return 0;
}

size_t stats_smem(int N, int nq, int nt, int ng)
{
#define X(n) if (N == n) return smem_stats<n>(nq, nt, ng);
    ENS_SUPPORTED_N(X)
#undef X
    return 0;
}

int stats_blocks(int N)
{
#define X(n) if (N == n) return stats_ctas<n>();
    ENS_SUPPORTED_N(X)
#undef X
    return 0;
}

const SizedOps *sized_ops(int N)
{
#define X(n) if (N == n) return sized_ops_for<n>();
    ENS_SUPPORTED_N(X)
#undef X
    return nullptr;
}

cudaError_t prepare_kernels(int N, int nq, int nt, int ng)
{
    const SizedOps *o = sized_ops(N);
    return o ? o->prepare(nq, nt, ng) : cudaErrorInvalidValue;
}

bool plan_variant_available(int N) { return has_plan_variant(N); }

int znl_ctas_per_sm(int N, int var)
{
    const SizedOps *o = sized_ops(N);
    return o ? o->znl_ctas_per_sm(var) : 0;
}

bool zplan_variant_available(int N) { return has_zplan_variant(N); }

bool fx_ws_available(int N)
{
    const SizedOps *o = sized_ops(N);
    return o && o->fx_ws();
}

void launch_pass(Pass pass, int mode, const Geo &g, MemberDev *md, const HistDev *h, int stage, int last, int arg,
                 cudaStream_t s)
{
    if (const SizedOps *o = sized_ops(g.N)) o->launch(pass, mode, g, md, h, stage, last, arg, s);
}

void launch_state_sums(const Geo &g, MemberDev *md, cudaStream_t s)
{
    const int ncols = g.NK * g.NZp;
    dim3 grid((ncols + 127) / 128, g.members);
    k_state_sums<<<grid, 128, 0, s>>>(g, md);
}

void launch_finish(MemberDev *md, int nmembers, const double *partial, int partial_blocks, int stage, int last,
                   int mode, cudaStream_t s)
{
    k_finish<<<nmembers, 32, 0, s>>>(md, partial, partial_blocks, stage, last, mode);
}

void launch_ic(const Geo &g, MemberDev *md, cudaStream_t s)
{
    // white noise -> forward along z, y, x with projection and shell sums
    cudaMemsetAsync(g.shell, 0, sizeof(double) * g.shells * g.members, s);
    launch_pass(Pass::Z, 1, g, md, nullptr, 0, 0, 0, s);
    launch_pass(Pass::FY, 0, g, md, nullptr, 0, 0, 0, s);
    launch_pass(Pass::FX, 2, g, md, nullptr, 0, 0, 0, s);
    k_ic_factors<<<g.members, 128, 0, s>>>(md, g);
    const long long modes = (long long)g.NK * g.NK * g.NZp;
    dim3 grid((unsigned)((modes + 255) / 256), g.members);
    k_ic_scale<<<grid, 256, 0, s>>>(g);
}

void launch_twiddles(float2 *tw, int N, cudaStream_t s) { k_twiddles<<<(N + 255) / 256, 256, 0, s>>>(tw, N); }

void launch_edges(float *eq, float *er, float *et, float *eg, int nq, int nt, int ng, double q_lim, double r_lim,
                  double t_lo, double t_hi, double g_lim, cudaStream_t s)
{
    k_edges<<<1, 256, 0, s>>>(eq, er, et, eg, nq, nt, ng, q_lim, r_lim, t_lo, t_hi, g_lim);
}

// the statistics pass's bin rule alone, on values already in an axis's
// units (0 Q, 1 R, 2 log10 tail, 3 gradient component), edges in global
// memory: the device functions k_z_stats calls per point
__global__ void k_bin_check(HistDev h, int axis, const float *__restrict__ x, int n, int *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = x[i];
    int b;
    if (axis == 0) b = bin_lin(v, lin_map(h.q_lo, h.q_inv_w), h.edges_q, h.nq);
    else if (axis == 1) b = bin_lin(v, lin_map(h.r_lo, h.r_inv_w), h.edges_r, h.nq);
    else if (axis == 2) b = bin_log(v, log_map(h.t_lo, h.t_inv_w), h.edges_t, h.nt);
    else b = bin_lin(v, lin_map(h.g_lo, h.g_inv_w), h.edges_g, h.ng);
    out[i] = b;
}

void launch_bin_check(const HistDev &h, int axis, const float *x, int n, int *out, cudaStream_t s)
{
    if (n > 0) k_bin_check<<<(n + 255) / 256, 256, 0, s>>>(h, axis, x, n, out);
}

void launch_finish_stats(const double *mom_partial, int blocks, double *moments, int nmembers, int accumulate,
                         cudaStream_t s)
{
    k_finish_stats<<<nmembers, 64, 0, s>>>(mom_partial, blocks, moments, accumulate);
}

void launch_mixture(const double *lam, int n, const MixWeightArgs &wa, const unsigned long long *counts,
                    const double *moments, const MixPdfArgs &pa, double *w, double *covered, double *pdf,
                    double *mom_mix, double *ratios, cudaStream_t s)
{
    k_mix_weights<<<1, 1024, 0, s>>>(lam, n, wa, w, covered);
    const int nb = mix_pdf_len(pa);
    k_mix_pdf<<<(nb + 255) / 256, 256, 0, s>>>(counts, moments, w, n, pa, pdf, mom_mix);
    k_mix_ratios<<<1, 32, 0, s>>>(mom_mix, ratios);
}

}  // namespace ens
