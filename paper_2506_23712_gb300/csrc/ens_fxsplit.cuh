// The last pass of an RK stage split in two launches (an autotuner variant
// of the fused k_fwd_x MODE 0):
//
//   k_fwd_x_fft : forward transform along x of the three n fields of buffer
//                 A, the kept kx rows written unscaled into the compact
//                 spectral layout [3][kx NK][ky NK][kz NZp] (in buffer A,
//                 from field 3 on, free at this point of the stage)
//   k_update    : per kept mode, 1/N^3, Leray projection, constant-power band
//                 forcing, integrating-factor RK stage and the FP64 partial
//                 sums of E, dissipation and band energy (Sec. IV)
//
// The split moves 2 x 3 compact fields more through HBM than the fused pass,
// but each launch is light (no staged tile, more resident warps); the
// arithmetic per mode is the fused pass's, in the same order.
#pragma once

#include "ens_kernels.cuh"

namespace ens {

template <int N>
__device__ __forceinline__ float2 *nhat_of(const Geo &g, int m)
{
    return g.A + ((long long)m * kFields + 3) * Dims<N>::SA;
}

// grid (NK*NZp/T, 3, members), block T*P
template <int N, int T>
__global__ void __launch_bounds__(ColCfg<N, T>::threads)
k_fwd_x_fft(Geo g)
{
    using PI = PlanInfo<N>;
    constexpr int P = PI::P, V = PI::V;
    extern __shared__ __align__(16) float2 sm[];
    float2 *tw = sm, *buf = sm + N;
    load_twiddles(tw, g.tw, N);
    const int c = threadIdx.x % T, p = threadIdx.x / T;
    const int q = blockIdx.y, m = blockIdx.z;
    const int col = blockIdx.x * T + c;                  // (ky, kz) flat
    const int iy = col / Dims<N>::NZP, kz = col % Dims<N>::NZP;
    const bool valid = kz < Dims<N>::NZ;
    const float2 *src = g.A + ((long long)m * kFields + q) * Dims<N>::SA + ((long long)iy * N) * Dims<N>::NZP + kz;
    float2 *dst = nhat_of<N>(g, m) + q * Dims<N>::SU + col;
    constexpr long long rowU = (long long)Dims<N>::NK * Dims<N>::NZP;
    float2 v[V];
#pragma unroll
    for (int i = 0; i < V; ++i) v[i] = valid ? src[(long long)PI::in_pos(p, i) * Dims<N>::NZP] : make_float2(0.f, 0.f);
    fft_line<N, true>(v, p, tw, [&](int pos) { return &buf[pos * T + c]; });
    if (valid) {
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const int kx = wnum(PI::out_pos(p, i), N);
            if (kx >= -Dims<N>::KC && kx <= Dims<N>::KC) dst[(kx >= 0 ? kx : kx + Dims<N>::NK) * rowU] = v[i];
        }
    }
}

constexpr int kUpdThreads = 256;
constexpr int kUpdModes = kUpdChunk / kUpdThreads;   // modes per thread

template <int N>
constexpr int update_blocks()
{
    return (int)((Dims<N>::SU + (long long)kUpdThreads * kUpdModes - 1) / ((long long)kUpdThreads * kUpdModes));
}

// grid (update_blocks<N>(), members), block kUpdThreads
template <int N>
__global__ void __launch_bounds__(kUpdThreads)
k_update(Geo g, MemberDev *md, int stage, int last_stage)
{
    __shared__ double scratch[(kUpdThreads / 32) * 3];
    const int m = blockIdx.y;
    const MemberDev &d = md[g.first + m];
    const float inv_n3 = 1.0f / ((float)N * (float)N * (float)N);
    const float dtf = (float)member_dt(d, N);
    const float alpha = (float)d.alpha;
    const float nu = (float)d.nu;
    const StageCoef co = stage_coef(d.rk, stage);
    const int blo = d.band_lo2, bhi = d.band_hi2;
    const float2 *nh = nhat_of<N>(g, m);
    float2 *U = g.U + (long long)m * 3 * Dims<N>::SU;
    float2 *S = g.S + (long long)m * 3 * Dims<N>::SU;
    float2 *dst = last_stage ? U : S;
    constexpr long long rowU = (long long)Dims<N>::NK * Dims<N>::NZP;
    float se = 0.f, sd = 0.f, sb = 0.f;
    const long long first = (long long)blockIdx.x * kUpdThreads * kUpdModes + threadIdx.x;
#pragma unroll
    for (int u = 0; u < kUpdModes; ++u) {
        const long long mi = first + (long long)u * kUpdThreads;
        if (mi >= Dims<N>::SU) break;
        const int ix = (int)(mi / rowU);
        const int rem = (int)(mi % rowU);
        const int iy = rem / Dims<N>::NZP, kz = rem % Dims<N>::NZP;
        if (kz >= Dims<N>::NZ) continue;
        const int kx = ix <= Dims<N>::KC ? ix : ix - Dims<N>::NK;
        const int ky = iy <= Dims<N>::KC ? iy : iy - Dims<N>::NK;
        const float fk[3] = {(float)kx, (float)ky, (float)kz};
        const int k2i = kx * kx + ky * ky + kz * kz;
        const float k2 = (float)k2i;
        float2 n[3], un[3], us[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            n[q] = cscale(nh[q * Dims<N>::SU + mi], inv_n3);
            un[q] = U[q * Dims<N>::SU + mi];
            us[q] = stage != 0 ? S[q * Dims<N>::SU + mi] : un[q];
        }
        // Leray projection P_ij = delta_ij - k_i k_j / k^2; k = 0 held at zero
        if (k2i == 0) {
            n[0] = n[1] = n[2] = make_float2(0.f, 0.f);
        } else {
            const float inv = 1.f / k2;
            const float dr = (fk[0] * n[0].x + fk[1] * n[1].x + fk[2] * n[2].x) * inv;
            const float di = (fk[0] * n[0].y + fk[1] * n[1].y + fk[2] * n[2].y) * inv;
#pragma unroll
            for (int q = 0; q < 3; ++q) n[q] = make_float2(n[q].x - fk[q] * dr, n[q].y - fk[q] * di);
        }
        const float wgt = kz == 0 ? 1.f : 2.f;   // Hermitian multiplicity in the full spectrum
        const bool band = k2i >= blo && k2i <= bhi;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (band) n[q] = make_float2(n[q].x + alpha * us[q].x, n[q].y + alpha * us[q].y);
        const float ea = co.a != 0.f ? expf(-nu * k2 * co.ha * dtf) : 0.f;
        const float eb = expf(-nu * k2 * co.hb * dtf);
        float a2 = 0.f;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float rx = us[q].x + dtf * n[q].x, ry = us[q].y + dtf * n[q].y;
            const float ox = co.a * ea * un[q].x + co.b * eb * rx;
            const float oy = co.a * ea * un[q].y + co.b * eb * ry;
            dst[q * Dims<N>::SU + mi] = make_float2(ox, oy);
            a2 += ox * ox + oy * oy;
        }
        se += 0.5f * wgt * a2;
        sd += nu * k2 * wgt * a2;
        if (band) sb += 0.5f * wgt * a2;
    }
    double vals[3] = {(double)se, (double)sd, (double)sb};
    double *out = g.partial + ((long long)(g.first + m) * g.partial_blocks + blockIdx.x) * 4;
    block_sum_to<3>(out, vals, scratch);
}

}  // namespace ens
