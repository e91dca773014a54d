// The last pass of an RK stage with its two halves overlapped inside an SM
// (an autotuner variant of the fused k_fwd_x MODE 0): forward transform along
// x, 1/N^3, Leray projection, constant-power band forcing, integrating-factor
// RK stage and the FP64 partial sums (Sec. IV).
//
// Persistent CTAs (one per SM) of two warp groups over 16-column tiles:
//   transform group : the three forward-x transforms of a tile into one of
//                     two shared-memory tile buffers (kept kx rows only)
//   update group    : per kept mode of the other buffer's tile, the stage
//                     update against the state rows U (and S), which it
//                     starts loading before the tile is ready
// The groups hand the buffers over with hardware named barriers (FULL[b]:
// transform arrives, update waits; EMPTY[b]: the reverse), so the update of
// tile k runs while tile k + 1 is transformed: the state reads overlap the
// transforms instead of following them, and no intermediate spectrum goes
// through HBM.  The arithmetic per mode and the partial-sum order are those
// of the fused pass with 16-column tiles (bit for bit the same fields and
// sums); every tile writes its partial sums into slot bx as that pass does.
#pragma once

#include "ens_kernels.cuh"

namespace ens {

template <int N>
struct WsCfg {
    static constexpr int T = 16;
    using PI = PlanInfo<N, 0>;
    static constexpr int TH = T * PI::P;                  // threads per group
    static constexpr int PER = Dims<N>::NK * T;           // kept modes of a tile per component
    static constexpr int TILES = Dims<N>::NK * Dims<N>::NZP / T;   // tiles per member
    static constexpr size_t smem() { return sizeof(float2) * ((size_t)N + (size_t)N * T + 2 * 3 * (size_t)PER); }
};

template <int N>
constexpr bool has_fx_ws() { return WsCfg<N>::TH == 256 && WsCfg<N>::smem() <= 220 * 1024; }

__device__ __forceinline__ void named_arrive(int id, int count)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// barrier IDs: 1, 2 FULL[b]; 3, 4 EMPTY[b]; 5 transform group; 6 update group
template <int N>
__global__ void __launch_bounds__(2 * WsCfg<N>::TH, 1)
k_fwd_x_ws(Geo g, MemberDev *md, int stage, int last_stage)
{
    using C = WsCfg<N>;
    using PI = typename C::PI;
    constexpr int T = C::T, P = PI::P, V = PI::V, TH = C::TH, PER = C::PER;
    extern __shared__ __align__(16) float2 sm[];
    __shared__ double red[(TH / 32) * 3];
    float2 *tw = sm, *buf = sm + N, *tiles = buf + N * T;   // tiles: [2][3][NK][T]
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = g.tw[i];
    __syncthreads();
    const long long ntiles = (long long)C::TILES * g.members;
    const int nk = ntiles > blockIdx.x ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x) + 1 : 0;   // tiles of this CTA
    const int lt = threadIdx.x % TH;
    if (threadIdx.x < TH) {
        // ---- transform group ----
        const int c = lt % T, p = lt / T;
        auto at = [&](int pos) { return &buf[pos * T + c]; };
        for (int k = 0; k < nk; ++k) {
            const long long t = blockIdx.x + (long long)k * gridDim.x;
            const int m = (int)(t / C::TILES), bx = (int)(t % C::TILES);
            float2 *tile = tiles + (k & 1) * 3 * PER;
            const int col = bx * T + c;                   // (ky, kz) flat
            const int iy = col / Dims<N>::NZP, kz = col % Dims<N>::NZP;
            const bool valid = kz < Dims<N>::NZ;
            const float2 *Ain = g.A + (long long)m * kFields * Dims<N>::SA + ((long long)iy * N) * Dims<N>::NZP + kz;
            float2 v[V], nxt[V];
#pragma unroll
            for (int i = 0; i < V; ++i)
                v[i] = valid ? Ain[(long long)PI::in_pos(p, i) * Dims<N>::NZP] : make_float2(0.f, 0.f);
            named_sync(3 + (k & 1), 2 * TH);   // EMPTY: the update group is done with this buffer
#pragma unroll 1
            for (int q = 0; q < 3; ++q) {
                if (q < 2) {
#pragma unroll
                    for (int i = 0; i < V; ++i)
                        nxt[i] = valid ? Ain[(long long)(q + 1) * Dims<N>::SA + (long long)PI::in_pos(p, i) * Dims<N>::NZP]
                                       : make_float2(0.f, 0.f);
                }
                fft_line<N, true, 0>(v, p, tw, at, NamedSync<5, TH>());
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const int kx = wnum(PI::out_pos(p, i), N);
                    if (kx >= -Dims<N>::KC && kx <= Dims<N>::KC)
                        tile[q * PER + (kx >= 0 ? kx : kx + Dims<N>::NK) * T + c] = v[i];
                }
                if (q < 2) {
#pragma unroll
                    for (int i = 0; i < V; ++i) v[i] = nxt[i];
                }
            }
            named_arrive(1 + (k & 1), 2 * TH);   // FULL
        }
    } else {
        // ---- update group ----
        if (nk > 0) named_arrive(3, 2 * TH);   // both buffers start empty
        if (nk > 1) named_arrive(4, 2 * TH);
        const int wg = lt >> 5;
        for (int k = 0; k < nk; ++k) {
            const long long t = blockIdx.x + (long long)k * gridDim.x;
            const int m = (int)(t / C::TILES), bx = (int)(t % C::TILES);
            const float2 *tile = tiles + (k & 1) * 3 * PER;
            const int col0 = bx * T;
            const int iy = col0 / Dims<N>::NZP;
            const int kz0 = col0 % Dims<N>::NZP;
            const MemberDev &d = md[g.first + m];
            const float inv_n3 = 1.0f / ((float)N * (float)N * (float)N);
            const long long rowU = (long long)Dims<N>::NK * Dims<N>::NZP;
            float2 *U = g.U + (long long)m * 3 * Dims<N>::SU + col0;
            float2 *S = g.S + (long long)m * 3 * Dims<N>::SU + col0;
            const int kyi = iy <= Dims<N>::KC ? iy : iy - Dims<N>::NK;
            const float dtf = (float)member_dt(d, N);
            const float alpha = (float)d.alpha, nu = (float)d.nu;
            const StageCoef co = stage_coef(d.rk, stage);
            const int blo = d.band_lo2, bhi = d.band_hi2;
            float se = 0.f, sd = 0.f, sb = 0.f;
            constexpr int UB = 4;
            bool waited = false;
            for (int base = lt; base < PER; base += UB * TH) {
                float2 unb[UB][3], usb[UB][3];
#pragma unroll
                for (int u = 0; u < UB; ++u) {
                    const int idx = base + u * TH;
                    const int cc = idx % T;
                    const bool ok = idx < PER && kz0 + cc < Dims<N>::NZ;
                    const long long off = (long long)(idx / T) * rowU + cc;
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        unb[u][q] = ok ? U[q * Dims<N>::SU + off] : make_float2(0.f, 0.f);
                        usb[u][q] = (ok && stage != 0) ? S[q * Dims<N>::SU + off] : unb[u][q];
                    }
                }
                if (!waited) {   // the first state rows are in flight: now wait for the tile
                    named_sync(1 + (k & 1), 2 * TH);
                    waited = true;
                }
#pragma unroll
                for (int u = 0; u < UB; ++u) {
                    const int idx = base + u * TH;
                    if (idx >= PER) continue;
                    const int ix = idx / T, cc = idx % T;
                    const int kzc = kz0 + cc;
                    if (kzc >= Dims<N>::NZ) continue;
                    const int kx = ix <= Dims<N>::KC ? ix : ix - Dims<N>::NK;
                    const float fk[3] = {(float)kx, (float)kyi, (float)kzc};
                    const int k2i = kx * kx + kyi * kyi + kzc * kzc;
                    const float k2 = (float)k2i;
                    const long long off = ix * rowU + cc;
                    float2 n[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) n[q] = cscale(tile[q * PER + idx], inv_n3);
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
                    const float wgt = kzc == 0 ? 1.f : 2.f;   // Hermitian multiplicity in the full spectrum
                    const bool band = k2i >= blo && k2i <= bhi;
                    float2 us[3], un[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        un[q] = unb[u][q];
                        us[q] = usb[u][q];
                        if (band) n[q] = make_float2(n[q].x + alpha * us[q].x, n[q].y + alpha * us[q].y);
                    }
                    const IfCoef ic = if_coef(co, nu, k2, dtf);
                    float2 *dst = last_stage ? U : S;
                    float a2 = 0.f;
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const float rx = us[q].x + dtf * n[q].x, ry = us[q].y + dtf * n[q].y;
                        const float ox = if_combine(ic, un[q].x, rx);
                        const float oy = if_combine(ic, un[q].y, ry);
                        dst[q * Dims<N>::SU + off] = make_float2(ox, oy);
                        a2 += ox * ox + oy * oy;
                    }
                    se += 0.5f * wgt * a2;
                    sd += nu * k2 * wgt * a2;
                    if (band) sb += 0.5f * wgt * a2;
                }
            }
            if (!waited) named_sync(1 + (k & 1), 2 * TH);
            // the tile buffer is free once every update thread is past its reads
            if (k + 2 < nk) named_arrive(3 + (k & 1), 2 * TH);
            // partial sums of the tile (the order of the fused pass's block reduction)
            double vals[3] = {(double)se, (double)sd, (double)sb};
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                double x = vals[q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                vals[q] = x;
            }
            if ((lt & 31) == 0) {
#pragma unroll
                for (int q = 0; q < 3; ++q) red[wg * 3 + q] = vals[q];
            }
            named_sync(6, TH);
            if (lt < 3) {
                double s = 0.0;
                for (int w = 0; w < TH / 32; ++w) s += red[w * 3 + lt];
                g.partial[((long long)(g.first + m) * g.partial_blocks + bx) * 4 + lt] = s;
            }
            named_sync(6, TH);   // red is rewritten by the next tile
        }
    }
}

}  // namespace ens
