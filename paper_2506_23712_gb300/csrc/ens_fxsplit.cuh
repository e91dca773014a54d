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
constexpr int kUpdPairs = kUpdChunk / (2 * kUpdThreads);   // mode pairs per thread

template <int N>
constexpr int update_blocks()
{
    return (int)((Dims<N>::SU + kUpdChunk - 1) / kUpdChunk);
}

// the update of one kept mode (Sec. IV): Leray projection of the nonlinear
// term, band forcing, one integrating-factor RK stage; returns |u|^2 of the
// result (both Hermitian halves counted by the caller)
struct UpdCoef {
    float inv_n3, dtf, alpha, nu, a, b, ha, hb;
    int blo, bhi;
};

__device__ __forceinline__ float update_mode(const UpdCoef &c, int kx, int ky, int kz, float2 (&n)[3],
                                             const float2 (&un)[3], const float2 (&us)[3], float2 (&out)[3],
                                             bool &band, float &k2out)
{
    const float fk[3] = {(float)kx, (float)ky, (float)kz};
    const int k2i = kx * kx + ky * ky + kz * kz;
    const float k2 = (float)k2i;
#pragma unroll
    for (int q = 0; q < 3; ++q) n[q] = cscale(n[q], c.inv_n3);
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
    band = k2i >= c.blo && k2i <= c.bhi;
#pragma unroll
    for (int q = 0; q < 3; ++q)
        if (band) n[q] = make_float2(n[q].x + c.alpha * us[q].x, n[q].y + c.alpha * us[q].y);
    const IfCoef ic = if_coef(StageCoef{c.a, c.ha, c.b, c.hb}, c.nu, k2, c.dtf);
    float a2 = 0.f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float rx = us[q].x + c.dtf * n[q].x, ry = us[q].y + c.dtf * n[q].y;
        const float ox = if_combine(ic, un[q].x, rx);
        const float oy = if_combine(ic, un[q].y, ry);
        out[q] = make_float2(ox, oy);
        a2 += ox * ox + oy * oy;
    }
    k2out = k2;
    return a2;
}

// grid (update_blocks<N>(), members), block kUpdThreads.  Thread t takes
// the mode pairs (2j, 2j + 1), j = first + t + u * kUpdThreads: 16-byte
// loads and stores, and every load of a pair issued before its arithmetic.
// A pair never straddles a kz row (NZp is even); a mode past the kept kz
// (odd NZ) is written as zero, a pair wholly past it is not touched.
template <int N>
__global__ void __launch_bounds__(kUpdThreads, 4)
k_update(Geo g, MemberDev *md, int stage, int last_stage)
{
    using D = Dims<N>;
    static_assert(D::NZP % 2 == 0 && D::SU % 2 == 0, "mode pairs must not straddle a row");
    __shared__ double scratch[(kUpdThreads / 32) * 3];
    const int m = blockIdx.y;
    const MemberDev &d = md[g.first + m];
    const StageCoef co = stage_coef(d.rk, stage);
    UpdCoef c;
    c.inv_n3 = 1.0f / ((float)N * (float)N * (float)N);
    c.dtf = (float)member_dt(d, N);
    c.alpha = (float)d.alpha;
    c.nu = (float)d.nu;
    c.a = co.a;
    c.b = co.b;
    c.ha = co.ha;
    c.hb = co.hb;
    c.blo = d.band_lo2;
    c.bhi = d.band_hi2;
    const float4 *nh = reinterpret_cast<const float4 *>(nhat_of<N>(g, m));
    const float4 *U = reinterpret_cast<const float4 *>(g.U + (long long)m * 3 * D::SU);
    const float4 *S = reinterpret_cast<const float4 *>(g.S + (long long)m * 3 * D::SU);
    float4 *dst = reinterpret_cast<float4 *>((last_stage ? g.U : g.S) + (long long)m * 3 * D::SU);
    constexpr long long rowU = (long long)D::NK * D::NZP;
    constexpr long long SU2 = D::SU / 2;   // pairs per component
    float se = 0.f, sd = 0.f, sb = 0.f;
    const long long first = (long long)blockIdx.x * (kUpdChunk / 2) + threadIdx.x;
#pragma unroll
    for (int u = 0; u < kUpdPairs; ++u) {
        const long long j = first + (long long)u * kUpdThreads;
        const long long mi = 2 * j;
        const int ix = (int)(mi / rowU);
        const int rem = (int)(mi % rowU);
        const int iy = rem / D::NZP, kz = rem % D::NZP;
        const bool any = j < SU2 && kz < D::NZ;
        const bool both = any && kz + 1 < D::NZ;
        float4 n4[3], u4[3], s4[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            n4[q] = any ? nh[q * SU2 + j] : z4;
            u4[q] = any ? U[q * SU2 + j] : z4;
            s4[q] = (any && stage != 0) ? S[q * SU2 + j] : u4[q];
        }
        if (!any) continue;
        const int kx = ix <= D::KC ? ix : ix - D::NK;
        const int ky = iy <= D::KC ? iy : iy - D::NK;
        float4 o4[3];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float2 n[3], un[3], us[3], o[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                n[q] = h ? make_float2(n4[q].z, n4[q].w) : make_float2(n4[q].x, n4[q].y);
                un[q] = h ? make_float2(u4[q].z, u4[q].w) : make_float2(u4[q].x, u4[q].y);
                us[q] = h ? make_float2(s4[q].z, s4[q].w) : make_float2(s4[q].x, s4[q].y);
            }
            bool band;
            float k2;
            const float a2 = update_mode(c, kx, ky, kz + h, n, un, us, o, band, k2);
            const bool keep = h == 0 || both;
            const float wgt = (kz + h) == 0 ? 1.f : 2.f;   // Hermitian multiplicity in the full spectrum
            if (keep) {
                se += 0.5f * wgt * a2;
                sd += c.nu * k2 * wgt * a2;
                if (band) sb += 0.5f * wgt * a2;
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float2 v = keep ? o[q] : make_float2(0.f, 0.f);
                if (h == 0) { o4[q].x = v.x; o4[q].y = v.y; } else { o4[q].z = v.x; o4[q].w = v.y; }
            }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) dst[q * SU2 + j] = o4[q];
    }
    double vals[3] = {(double)se, (double)sd, (double)sb};
    double *out = g.partial + ((long long)(g.first + m) * g.partial_blocks + blockIdx.x) * 4;
    block_sum_to<3>(out, vals, scratch);
}

}  // namespace ens
