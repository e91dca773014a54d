// Fused gradient-invariant + histogram + moment pass (sm_103a).
//
// Input: the eight independent velocity-gradient components A_ij = d_j u_i
// (ij = 11,12,13,21,22,23,31,32), already transformed along x and y (buffer
// B); A_33 = -A_11 - A_22 by incompressibility.  Per grid point:
//   Q = -1/2 Tr A^2, R = -1/3 Tr A^3            (Sec. V)
//   eps = 2 nu Tr S^2, omega^2 = |omega|^2       (Sec. VI)
// binned into the joint Q-R histogram (units q0 = eps_norm / (2 nu_norm)),
// log10 histograms of eps/eps_norm and omega^2 nu_norm/eps_norm and, when
// requested, linear histograms of the gradient components A_ij / sqrt(q0)
// (longitudinal and transverse pooled separately, Sec. VI).  Bin rule:
// bin b iff edge[b] <= x < edge[b+1] on FP32 edges (estimate from the affine
// or log10 map, then corrected against the edge table, so the decision is
// exactly the edge comparison).  Counts go to per-CTA shared-memory
// histograms with warp-aggregated increments (__match_any_sync), flushed to
// the member's uint64 counts once per CTA.  Moments: FP32 sums per thread
// over its points, warp shuffle reduction, FP64 accumulation per warp and
// per CTA, FP64 fixed-order reduction across CTAs.
#pragma once

#include "ens_kernels.cuh"

namespace ens {

__device__ __forceinline__ int bin_lin(float x, float lo, float inv_w, const float *e, int n)
{
    if (x < e[0]) return -1;
    if (x >= e[n]) return n;
    int b = (int)floorf((x - lo) * inv_w);
    b = min(max(b, 0), n - 1);
    while (b > 0 && e[b] > x) --b;
    while (b < n - 1 && e[b + 1] <= x) ++b;
    return b;
}

__device__ __forceinline__ int bin_log(float x, float lo, float inv_w, const float *e, int n)
{
    if (!(x > 0.f) || x < e[0]) return -1;
    if (x >= e[n]) return n;
    int b = (int)floorf((log10f(x) - lo) * inv_w);
    b = min(max(b, 0), n - 1);
    while (b > 0 && e[b] > x) --b;
    while (b < n - 1 && e[b + 1] <= x) ++b;
    return b;
}

// warp-aggregated increment of hist[key] (key < 0: no increment)
__device__ __forceinline__ void warp_count(unsigned *hist, int key)
{
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[key], (unsigned)__popc(peers));
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int N>
constexpr size_t smem_stats(int nq, int nt, int ng)
{
    return smem_rows<N>() + sizeof(unsigned) * (size_t)counts_len_of(nq, nt, ng) +
           sizeof(float) * (2 * (nq + 1) + nt + 1 + ng + 1) + sizeof(double) * 8 * kNMom + 64;
}

template <int N>
__global__ void __launch_bounds__(256, 1)
k_z_stats(Geo g, HistDev h, const MemberDev *md)
{
    using PI = WPlanInfo<N>;
    using RC = RowCfg<N>;
    constexpr int P = PI::P, V = PI::V, RZ = RC::RZ;
    extern __shared__ __align__(16) float2 sm[];
    float2 *tw = sm, *buf = sm + N;
    const int L = h.counts_len;
    unsigned *hist = reinterpret_cast<unsigned *>(buf + RZ * RC::SROW);
    float *eq = reinterpret_cast<float *>(hist + L);
    float *er = eq + (h.nq + 1);
    float *et = er + (h.nq + 1);
    float *eg = et + (h.nt + 1);
    double *wmom = reinterpret_cast<double *>(
        (reinterpret_cast<uintptr_t>(eg + h.ng + 1) + 15) & ~(uintptr_t)15);
    for (int i = threadIdx.x; i < L; i += blockDim.x) hist[i] = 0u;
    for (int i = threadIdx.x; i <= h.nq; i += blockDim.x) {
        eq[i] = h.edges_q[i];
        er[i] = h.edges_r[i];
    }
    for (int i = threadIdx.x; i <= h.nt; i += blockDim.x) et[i] = h.edges_t[i];
    for (int i = threadIdx.x; i <= h.ng && h.ng > 0; i += blockDim.x) eg[i] = h.edges_g[i];
    for (int i = threadIdx.x; i < 8 * kNMom; i += blockDim.x) wmom[i] = 0.0;
    load_twiddles(tw, g.tw, N);

    const int p = threadIdx.x % P, r = threadIdx.x / P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m = blockIdx.y;
    const float nu = (float)md[g.first + m].nu;
    const long long nrows = (long long)N * N;
    auto at = [&](int pos) { return row_slot<N>(buf, r, pos); };
    const int off_e = h.nq * h.nq, off_w = off_e + h.nt, off_c = off_w + h.nt;
    const int off_gl = off_c + 8, off_gt = off_gl + h.ng, off_gc = off_gt + h.ng;
    int valid_rows = 0;

#pragma unroll 1
    for (int it = 0; it < kStatsIters; ++it) {
        const long long rho = ((long long)blockIdx.x * kStatsIters + it) * RZ + r;
        const bool row_ok = rho < nrows;
        if (threadIdx.x == 0) {
            const long long first_row = ((long long)blockIdx.x * kStatsIters + it) * RZ;
            valid_rows += (int)max(0LL, min((long long)RZ, nrows - first_row));
        }
        const float2 *B = g.B + (long long)m * kFields * Dims<N>::SB + (row_ok ? rho : 0) * Dims<N>::NZP;
        float2 v[4][V];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int i = 0; i < V; ++i)
                v[q][i] = row_ok ? pair_at(B + (2 * q) * Dims<N>::SB, B + (2 * q + 1) * Dims<N>::SB, PI::in_pos(p, i), N, Dims<N>::KC)
                                 : make_float2(0.f, 0.f);
            fft_line_warp<N, false>(v[q], p, tw, at);
        }
        float sQ = 0.f, sR = 0.f, sE = 0.f, sW = 0.f, sQ2 = 0.f, sR2 = 0.f, sE2 = 0.f, sW2 = 0.f;
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const float a11 = v[0][i].x, a12 = v[0][i].y, a13 = v[1][i].x, a21 = v[1][i].y;
            const float a22 = v[2][i].x, a23 = v[2][i].y, a31 = v[3][i].x, a32 = v[3][i].y;
            const float a33 = -a11 - a22;
            const float A[3][3] = {{a11, a12, a13}, {a21, a22, a23}, {a31, a32, a33}};
            float tr2 = 0.f, tr3 = 0.f;
#pragma unroll
            for (int ii = 0; ii < 3; ++ii)
#pragma unroll
                for (int jj = 0; jj < 3; ++jj) {
                    tr2 = fmaf(A[ii][jj], A[jj][ii], tr2);
                    float b = 0.f;   // (A^2)_ij
#pragma unroll
                    for (int kk = 0; kk < 3; ++kk) b = fmaf(A[ii][kk], A[kk][jj], b);
                    tr3 = fmaf(b, A[jj][ii], tr3);
                }
            const float s12 = 0.5f * (a12 + a21), s13 = 0.5f * (a13 + a31), s23 = 0.5f * (a23 + a32);
            const float ss = a11 * a11 + a22 * a22 + a33 * a33 + 2.f * (s12 * s12 + s13 * s13 + s23 * s23);
            const float wx = a32 - a23, wy = a13 - a31, wz = a21 - a12;
            const float Q = -0.5f * tr2, R = -tr3 * (1.f / 3.f);
            const float eps = 2.f * nu * ss, ens = wx * wx + wy * wy + wz * wz;
            if (row_ok) {
                sQ += Q; sR += R; sE += eps; sW += ens;
                sQ2 += Q * Q; sR2 += R * R; sE2 += eps * eps; sW2 += ens * ens;
            }
            const float xq = Q * h.q_scale, xr = R * h.r_scale, xe = eps * h.eps_scale, xw = ens * h.ens_scale;
            const bool finite = isfinite(xq) && isfinite(xr) && isfinite(xe) && isfinite(xw);
            int kq = -1, ke = -1, kw = -1;
            if (row_ok) {
                if (!finite) {
                    kq = off_c + 5;
                } else {
                    const int bq = bin_lin(xq, h.q_lo, h.q_inv_w, eq, h.nq);
                    const int br = bin_lin(xr, h.r_lo, h.r_inv_w, er, h.nq);
                    kq = (bq >= 0 && bq < h.nq && br >= 0 && br < h.nq) ? bq * h.nq + br : off_c + 0;
                    const int be = bin_log(xe, h.t_lo, h.t_inv_w, et, h.nt);
                    ke = be < 0 ? off_c + 1 : (be >= h.nt ? off_c + 2 : off_e + be);
                    const int bw = bin_log(xw, h.t_lo, h.t_inv_w, et, h.nt);
                    kw = bw < 0 ? off_c + 3 : (bw >= h.nt ? off_c + 4 : off_w + bw);
                }
            }
            warp_count(hist, kq);
            warp_count(hist, ke);
            warp_count(hist, kw);
            if (h.ng > 0) {
                // gradient components (longitudinal c = 0, 4, 8 pooled; the
                // six transverse ones pooled), finite points only
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    int kg = -1;
                    if (row_ok && finite) {
                        const float x = A[c / 3][c % 3] * h.g_scale;
                        const int bg = bin_lin(x, h.g_lo, h.g_inv_w, eg, h.ng);
                        const bool lon = c % 4 == 0;
                        kg = bg < 0 ? off_gc + (lon ? 0 : 2)
                                    : (bg >= h.ng ? off_gc + (lon ? 1 : 3) : (lon ? off_gl : off_gt) + bg);
                    }
                    warp_count(hist, kg);
                }
            }
        }
        // moments: sums of A_c^p (p = 2, 3, 4, 6) and of the invariants
        const float inv_vals[8] = {sQ, sR, sE, sW, sQ2, sR2, sE2, sW2};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float s = warp_sum(inv_vals[q]);
            if (lane == 0) wmom[warp * kNMom + 36 + q] += (double)s;
        }
#pragma unroll
        for (int comp = 0; comp < 9; ++comp) {
            float s2 = 0.f, s3 = 0.f, s4 = 0.f, s6 = 0.f;
            if (row_ok) {
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    float a;
                    switch (comp) {
                    case 0: a = v[0][i].x; break;
                    case 1: a = v[0][i].y; break;
                    case 2: a = v[1][i].x; break;
                    case 3: a = v[1][i].y; break;
                    case 4: a = v[2][i].x; break;
                    case 5: a = v[2][i].y; break;
                    case 6: a = v[3][i].x; break;
                    case 7: a = v[3][i].y; break;
                    default: a = -v[0][i].x - v[2][i].x; break;
                    }
                    const float a2 = a * a;
                    s2 += a2;
                    s3 = fmaf(a2, a, s3);
                    s4 = fmaf(a2, a2, s4);
                    s6 = fmaf(a2 * a2, a2, s6);
                }
            }
            s2 = warp_sum(s2);
            s3 = warp_sum(s3);
            s4 = warp_sum(s4);
            s6 = warp_sum(s6);
            if (lane == 0) {
                double *w = wmom + warp * kNMom + 4 * comp;
                w[0] += (double)s2;
                w[1] += (double)s3;
                w[2] += (double)s4;
                w[3] += (double)s6;
            }
        }
    }
    __syncthreads();
    unsigned long long *cnt = g.counts + (long long)(g.first + m) * L;
    for (int i = threadIdx.x; i < L; i += blockDim.x)
        if (hist[i]) atomicAdd(&cnt[i], (unsigned long long)hist[i]);
    if (threadIdx.x == 0) atomicAdd(&cnt[off_c + 6], (unsigned long long)valid_rows * N);
    if (threadIdx.x < kNMom) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wmom[w * kNMom + threadIdx.x];
        g.mom_partial[((long long)(g.first + m) * g.mom_blocks + blockIdx.x) * kNMom + threadIdx.x] = s;
    }
}

}  // namespace ens
