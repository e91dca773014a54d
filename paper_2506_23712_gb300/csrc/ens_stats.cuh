// Fused gradient-invariant + histogram + moment pass (sm_103a).
//
// Input: the eight independent velocity-gradient components A_ij = d_j u_i
// (ij = 11,12,13,21,22,23,31,32), already transformed along x and y (buffer
// B); A_33 = -A_11 - A_22 by incompressibility.  Per grid point:
//   Q = -1/2 Tr A^2, R = -1/3 Tr A^3 = -det A   (Sec. V; A traceless)
//   eps = 2 nu Tr S^2, omega^2 = |omega|^2       (Sec. VI)
// binned into the joint Q-R histogram (units q0 = eps_norm / (2 nu_norm)),
// log10 histograms of eps/eps_norm and omega^2 nu_norm/eps_norm and, when
// requested, linear histograms of the gradient components A_ij / sqrt(q0)
// (longitudinal and transverse pooled separately, Sec. VI).  Bin rule:
// bin b iff edge[b] <= x < edge[b+1] on FP32 edges (the floor of the affine
// or log map's estimate, corrected once against the edge table, so the
// decision is exactly the edge comparison).  Counts go to per-CTA shared-memory
// histograms (plain shared atomics for the Q-R and tail histograms,
// warp-aggregated increments for the gradient components), flushed to the
// member's uint64 counts once per CTA.  Moments: FP32 sums per thread
// (packed FP32x2 for the component pairs) over up to kStatsFlush rows, warp
// shuffle reduction into FP64 per warp, FP64 fixed-order reduction across
// warps and CTAs.
//
// Layout of the work: grid (stats_ctas<N>(), members); CTA c of member m
// takes a contiguous block of rows, its warps stream over the row groups of
// the block (32/P rows per group).  A warp stages the eight half-spectrum
// rows of a group in shared memory (cp.async.bulk, TMA; zero past the kept
// modes), reads them into registers, and refills the same buffer with the
// next group while it transforms and bins the current one (the work per
// group far outlasts the copy); the four Hermitian pair lines go to physical
// space with the z pass's warp-local transforms, their twiddles read from a
// lane-major shared table (registers go to more resident warps).
#pragma once

#include "ens_kernels.cuh"
#include "ens_tma.cuh"
#include "ens_znl.cuh"

namespace ens {

// Bin of x from its estimated bin coordinate t (affine or log map, within
// far less than one bin of the exact position): the floor of t, clamped to
// the table, then one correction against the FP32 edges, so the decision is
// exactly edge[b] <= x < edge[b + 1]; -1 below edge[0] (x <= 0 for a log
// map), n at or above edge[n].  Branch-free: no lane of a warp waits on
// another's edge case.
__device__ __forceinline__ int bin_tab(float x, float t, const float *e, int n)
{
    int b = __float2int_rd(t);
    b = min(max(b, 0), n - 1);
    return b + (x >= e[b + 1] ? 1 : 0) - (x < e[b] ? 1 : 0);
}

// Estimate maps in one FMA each: (x - lo) / w as x a + c, log10(x) -
// lo over w as log2(x) a + c (the edge comparison decides)
struct BinMap {
    float a, c;
};
__device__ __forceinline__ BinMap lin_map(float lo, float inv_w) { return {inv_w, -lo * inv_w}; }
__device__ __forceinline__ BinMap log_map(float lo, float inv_w) { return {0.30102999566f * inv_w, -lo * inv_w}; }

__device__ __forceinline__ int bin_lin(float x, BinMap m, const float *e, int n)
{
    return bin_tab(x, fmaf(x, m.a, m.c), e, n);
}

// log10 bins from the hardware log2
__device__ __forceinline__ int bin_log(float x, BinMap m, const float *e, int n)
{
    return bin_tab(x, fmaf(__log2f(x), m.a, m.c), e, n);
}

// increment of hist[key] without aggregation (key < 0: none)
__device__ __forceinline__ void lane_count(unsigned *hist, int key)
{
    if (key >= 0) atomicAdd(&hist[key], 1u);
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

// Shape of the statistics pass: warps per CTA, staged row pitch, CTAs per member.
template <int N>
struct SCfg {
    using PI = WPlanInfo<N>;
    static constexpr int P = PI::P, V = PI::V, LPW = 32 / P;
    static constexpr int NZ2 = (kc_of_n(N) + 2) / 2 * 2;     // copied row length (16-byte multiple)
    static constexpr int PITCH = stage_pitch<N, 0>();        // staged row pitch, zero past NZ2
    static constexpr int STAGE = LPW * 8 * PITCH;            // float2 per warp (one buffer)
    static constexpr bool PAD = WPad<N>::on;
    static constexpr int SROW = PAD ? WPad<N>::SROW : RowCfg<N>::SROW;
    // warps per CTA: 12 where the plan's four lines fit the register share
    // of 12 resident warps, 8 for the 12- and 16-value plans (384, 512); 16
    // at 256 (128 registers with a few spilled: 24.7 against 25.1 ms per
    // 64-member snapshot; 14 warps, unevenly spread over the four schedulers,
    // 26.3 ms)
    static constexpr int WPB = V > 8 ? 8 : (N == 256 ? 16 : 12);
    static constexpr int GROUPS = N * N / LPW;               // row groups per member
    static constexpr int LT = PAD ? (LaneTw<N>::SIZE + 1) / 2 * 2 : 0;   // lane-major twiddles (float2)
    // CTAs per member: a power of two up to 32, at least 32 row groups per warp
    static constexpr int pow2_floor(int x) { return x >= 32 ? 32 : x >= 16 ? 16 : x >= 8 ? 8 : x >= 4 ? 4 : x >= 2 ? 2 : 1; }
    static constexpr int CTAS = pow2_floor(GROUPS / (WPB * 32));
    static_assert(GROUPS % CTAS == 0, "row groups split evenly over the CTAs of a member");
};

// moment partials are flushed from FP32 registers to FP64 every kStatsFlush row groups
constexpr int kStatsFlush = 32;

template <int N>
constexpr int stats_ctas() { return SCfg<N>::CTAS; }

template <int N>
constexpr size_t smem_stats(int nq, int nt, int ng)
{
    using C = SCfg<N>;
    return sizeof(float2) * (size_t)(N + C::LT) + sizeof(uint64_t) * 2 * C::WPB + sizeof(float2) * (size_t)C::WPB * C::STAGE +
           sizeof(float2) * (size_t)C::WPB * C::LPW * C::SROW + sizeof(double) * C::WPB * kNMom +
           sizeof(unsigned) * (size_t)counts_len_of(nq, nt, ng) + sizeof(float) * (2 * (nq + 1) + nt + 1 + ng + 1) + 16;
}

// packed FP32x2 helpers for the moment sums
__device__ __forceinline__ float2 pmul(float2 a, float2 b)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2bits(a)), "l"(f2bits(b)));
    return bitsf2(r);
}
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2bits(a)), "l"(f2bits(b)), "l"(f2bits(c)));
    return bitsf2(r);
}

template <int N>
__global__ void __launch_bounds__(32 * SCfg<N>::WPB, 1)
k_z_stats(Geo g, HistDev h, const MemberDev *md)
{
    using C = SCfg<N>;
    using PI = WPlanInfo<N>;
    constexpr int P = C::P, V = C::V, LPW = C::LPW, NZ2 = C::NZ2, WPB = C::WPB;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *tw = reinterpret_cast<float2 *>(smraw);
    float2 *ltw = tw + N;   // lane-major inter-pass twiddles (padded plans)
    uint64_t *bars = reinterpret_cast<uint64_t *>(ltw + C::LT);
    float2 *stage = reinterpret_cast<float2 *>(bars + 2 * WPB);
    float2 *rows = stage + WPB * C::STAGE;
    double *wmom = reinterpret_cast<double *>(rows + WPB * LPW * C::SROW);
    unsigned *hist = reinterpret_cast<unsigned *>(wmom + WPB * kNMom);
    const int L = h.counts_len;
    float *eq = reinterpret_cast<float *>(hist + L);
    float *er = eq + (h.nq + 1);
    float *et = er + (h.nq + 1);
    float *eg = et + (h.nt + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int line = lane / P, p = lane % P;
    uint64_t *bar = bars + 2 * warp;
    float2 *st = stage + warp * C::STAGE;
    float2 *rowbuf = rows + warp * LPW * C::SROW;
    for (int i = threadIdx.x; i < L; i += blockDim.x) hist[i] = 0u;
    for (int i = threadIdx.x; i <= h.nq; i += blockDim.x) {
        eq[i] = h.edges_q[i];
        er[i] = h.edges_r[i];
    }
    for (int i = threadIdx.x; i <= h.nt; i += blockDim.x) et[i] = h.edges_t[i];
    for (int i = threadIdx.x; i <= h.ng && h.ng > 0; i += blockDim.x) eg[i] = h.edges_g[i];
    for (int i = threadIdx.x; i < WPB * kNMom; i += blockDim.x) wmom[i] = 0.0;
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        fence_mbar_init();
    }
    // zero tails of the staged rows (never written by the copies)
    constexpr int TAIL = C::PITCH - NZ2;
    if constexpr (TAIL > 0) {
        for (int e = lane; e < LPW * 8 * TAIL; e += 32) st[(e / TAIL) * C::PITCH + NZ2 + e % TAIL] = make_float2(0.f, 0.f);
    }
    if constexpr (C::PAD) LaneTw<N>::init(ltw, g.tw);
    load_twiddles(tw, g.tw, N);   // block barrier: tables, barrier init and tails published

    const int m = blockIdx.y;
    const float nu = (float)md[g.first + m].nu;
    constexpr int GPC = C::GROUPS / C::CTAS;   // row groups of this CTA
    const long long g0 = (long long)blockIdx.x * GPC;
    const uint32_t bytes = (uint32_t)(LPW * 8 * NZ2 * sizeof(float2));
    const float2 *Bm = g.B + (long long)m * kFields * Dims<N>::SB;
    auto issue = [&](int k) {   // lane 0: row group g0 + k
        const float2 *src = Bm + ((g0 + k) * LPW) * Dims<N>::NZP;
        float2 *dst = st;
        mbar_arrive_expect_tx(&bar[0], bytes);
#pragma unroll 1
        for (int l = 0; l < LPW; ++l)
#pragma unroll
            for (int f = 0; f < 8; ++f)
                bulk_g2s(dst + (l * 8 + f) * C::PITCH, src + f * Dims<N>::SB + l * Dims<N>::NZP,
                         NZ2 * (uint32_t)sizeof(float2), &bar[0]);
    };
    int k = warp;
    if (lane == 0 && k < GPC) issue(k);

    auto at = [&](int pos) { return row_slot<N>(rowbuf, line, pos); };
    float2 *myrow = rowbuf + line * C::SROW;
    const int off_e = h.nq * h.nq, off_w = off_e + h.nt, off_c = off_w + h.nt;
    const BinMap mq = lin_map(h.q_lo, h.q_inv_w), mr = lin_map(h.r_lo, h.r_inv_w);
    const BinMap mt = log_map(h.t_lo, h.t_inv_w), mg = lin_map(h.g_lo, h.g_inv_w);
    const int off_gl = off_c + 8, off_gt = off_gl + h.ng, off_gc = off_gt + h.ng;

    // FP32 moment partials: component pairs (2q, 2q + 1) packed, A_33 alone,
    // invariant sums
    float2 S2[4], S3[4], S4[4], S6[4];
    float T2, T3, T4, T6;
    float inv[8];
    auto zero = [&]() {
#pragma unroll
        for (int q = 0; q < 4; ++q) S2[q] = S3[q] = S4[q] = S6[q] = make_float2(0.f, 0.f);
        T2 = T3 = T4 = T6 = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) inv[q] = 0.f;
    };
    auto flush = [&]() {   // whole warp: FP32 partials -> FP64 per warp
        float vals[kNMom - 4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            vals[4 * (2 * q) + 0] = S2[q].x; vals[4 * (2 * q) + 1] = S3[q].x; vals[4 * (2 * q) + 2] = S4[q].x; vals[4 * (2 * q) + 3] = S6[q].x;
            vals[4 * (2 * q + 1) + 0] = S2[q].y; vals[4 * (2 * q + 1) + 1] = S3[q].y; vals[4 * (2 * q + 1) + 2] = S4[q].y; vals[4 * (2 * q + 1) + 3] = S6[q].y;
        }
        vals[32] = T2; vals[33] = T3; vals[34] = T4; vals[35] = T6;
#pragma unroll
        for (int q = 0; q < 8; ++q) vals[36 + q] = inv[q];
#pragma unroll
        for (int q = 0; q < kNMom - 4; ++q) {
            const float s = warp_sum(vals[q]);
            if (lane == 0) wmom[warp * kNMom + q] += (double)s;
        }
        zero();
    };
    zero();

    bool timed_out = false;
    int it = 0;
    for (; k < GPC; ++it, k += WPB) {
        if (!mbar_wait_warp(&bar[0], (uint32_t)(it & 1))) {
            timed_out = true;
            break;
        }
        const float2 *X = st + line * 8 * C::PITCH;
        constexpr int R = C::PITCH;
        float2 v[4][V];
#pragma unroll
        for (int q = 0; q < 4; ++q) PairSlots<N, 0, 0>::load(v[q], X + 2 * q * R, X + (2 * q + 1) * R, p);
        __syncwarp();   // staged rows read: the buffer takes the next group
        if (lane == 0 && k + WPB < GPC) {
            fence_proxy_async_smem();   // the reads above precede the refill
            issue(k + WPB);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if constexpr (C::PAD) fft_line_warp_pad_lt<N, false>(v[q], p, ltw, myrow);
            else fft_line_warp<N, false>(v[q], p, tw, at);
        }
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const float a11 = v[0][i].x, a12 = v[0][i].y, a13 = v[1][i].x, a21 = v[1][i].y;
            const float a22 = v[2][i].x, a23 = v[2][i].y, a31 = v[3][i].x, a32 = v[3][i].y;
            const float a33 = -a11 - a22;
            // traceless A: Tr A^2 = sum_ij a_ij a_ji, Tr A^3 = 3 det A
            const float tr2 = a11 * a11 + a22 * a22 + a33 * a33 + 2.f * (a12 * a21 + a13 * a31 + a23 * a32);
            const float det = a11 * (a22 * a33 - a23 * a32) - a12 * (a21 * a33 - a23 * a31) + a13 * (a21 * a32 - a22 * a31);
            const float s12 = 0.5f * (a12 + a21), s13 = 0.5f * (a13 + a31), s23 = 0.5f * (a23 + a32);
            const float ss = a11 * a11 + a22 * a22 + a33 * a33 + 2.f * (s12 * s12 + s13 * s13 + s23 * s23);
            const float wx = a32 - a23, wy = a13 - a31, wz = a21 - a12;
            const float Q = -0.5f * tr2, R3 = -det;
            const float eps = 2.f * nu * ss, ens = wx * wx + wy * wy + wz * wz;
            inv[0] += Q; inv[1] += R3; inv[2] += eps; inv[3] += ens;
            inv[4] = fmaf(Q, Q, inv[4]); inv[5] = fmaf(R3, R3, inv[5]);
            inv[6] = fmaf(eps, eps, inv[6]); inv[7] = fmaf(ens, ens, inv[7]);
            const float xq = Q * h.q_scale, xr = R3 * h.r_scale, xe = eps * h.eps_scale, xw = ens * h.ens_scale;
            // Tr S^2 involves every component (a_33 and the symmetric
            // parts of all pairs), so it is finite exactly when A is
            const bool finite = isfinite(ss);
            // keys of all four lookups, then one select for a non-finite
            // point (its bins are meaningless but in the table's range)
            const int bq = bin_lin(xq, mq, eq, h.nq);
            const int br = bin_lin(xr, mr, er, h.nq);
            const int be = bin_log(xe, mt, et, h.nt);
            const int bw = bin_log(xw, mt, et, h.nt);
            int kq = ((unsigned)bq < (unsigned)h.nq && (unsigned)br < (unsigned)h.nq) ? bq * h.nq + br : off_c + 0;
            int ke = be < 0 ? off_c + 1 : (be >= h.nt ? off_c + 2 : off_e + be);
            int kw = bw < 0 ? off_c + 3 : (bw >= h.nt ? off_c + 4 : off_w + bw);
            if (!finite) {
                kq = off_c + 5;
                ke = kw = -1;
            }
            lane_count(hist, kq);
            lane_count(hist, ke);
            lane_count(hist, kw);
            if (h.ng > 0) {
                // gradient components (longitudinal c = 0, 4, 8 pooled; the
                // six transverse ones pooled), finite points only
                const float A[9] = {a11, a12, a13, a21, a22, a23, a31, a32, a33};
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    int kg = -1;
                    if (finite) {
                        const int bg = bin_lin(A[c] * h.g_scale, mg, eg, h.ng);
                        const bool lon = c % 4 == 0;
                        kg = bg < 0 ? off_gc + (lon ? 0 : 2)
                                    : (bg >= h.ng ? off_gc + (lon ? 1 : 3) : (lon ? off_gl : off_gt) + bg);
                    }
                    warp_count(hist, kg);
                }
            }
            // moments of the components: sums of A_c^p, p = 2, 3, 4, 6
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 a = v[q][i];
                const float2 a2 = pmul(a, a);
                const float2 a4 = pmul(a2, a2);
                S2[q] = cadd_x2(S2[q], a2);
                S3[q] = pfma(a2, a, S3[q]);
                S4[q] = cadd_x2(S4[q], a4);
                S6[q] = pfma(a4, a2, S6[q]);
            }
            const float b2 = a33 * a33;
            T2 += b2;
            T3 = fmaf(b2, a33, T3);
            T4 = fmaf(b2, b2, T4);
            T6 = fmaf(b2 * b2, b2, T6);
        }
        if ((it + 1) % kStatsFlush == 0) flush();
    }
    flush();
    if (timed_out) {
        if (lane == 0) atomicOr(const_cast<int *>(&md[g.first + m].flags), kFlagTimeout);
        mbar_wait_warp(&bar[0], (uint32_t)(it & 1));   // the copy in flight, once more (bounded)
    }
    __syncthreads();
    unsigned long long *cnt = g.counts + (long long)(g.first + m) * L;
    for (int i = threadIdx.x; i < L; i += blockDim.x)
        if (hist[i]) atomicAdd(&cnt[i], (unsigned long long)hist[i]);
    if (threadIdx.x == 0) atomicAdd(&cnt[off_c + 6], (unsigned long long)GPC * LPW * N);
    if (threadIdx.x < kNMom) {
        double s = 0.0;
        for (int w = 0; w < WPB; ++w) s += wmom[w * kNMom + threadIdx.x];
        g.mom_partial[((long long)(g.first + m) * g.mom_blocks + blockIdx.x) * kNMom + threadIdx.x] = s;
    }
}

}  // namespace ens
