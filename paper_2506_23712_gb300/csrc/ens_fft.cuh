// Register/shared-memory Stockham FFT engine for sm_103a.
//
// A length-N complex line is held by P threads, V = N/P values each.  A plan
// N = R0 * R1 (* R2) runs one radix-R pass per factor: every thread applies
// the inter-pass twiddles to its butterflies, computes R-point DFTs in
// registers, and hands the results to the next pass through shared memory
// (one exchange per pass boundary).  Pass s with radix R after Ns points of
// previous radices reads positions j + t N/R and writes position
// (j / Ns) Ns R + (j mod Ns) + t Ns (Stockham autosort: natural order out).
// The first pass's inputs come straight from global memory and the last
// pass's outputs go straight back, so a plan with two factors touches shared
// memory once.
//
// The transforms are the discrete Fourier series of the member fields
// (Sec. IV: the forcing acts on "velocity Fourier coefficients"); sign -1 is
// the analysis (forward) direction, +1 synthesis.  All arithmetic is FP32;
// twiddles come from an FP64-generated table rounded to FP32.
#pragma once

#include <cuda_runtime.h>

namespace ens {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// The same as one packed FP32x2 instruction (sm_100 family; both halves
// rounded to nearest, as the two scalar operations): half the issue slots.
// The line transforms take them where issue slots bound the kernel (PK).
__device__ __forceinline__ unsigned long long f2bits(float2 a) { return *reinterpret_cast<const unsigned long long *>(&a); }
__device__ __forceinline__ float2 bitsf2(unsigned long long r) { return *reinterpret_cast<const float2 *>(&r); }
__device__ __forceinline__ float2 cadd_x2(float2 a, float2 b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2bits(a)), "l"(f2bits(b)));
    return bitsf2(r);
}
__device__ __forceinline__ float2 csub_x2(float2 a, float2 b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2bits(a)), "l"(f2bits(b)));
    return bitsf2(r);
}
// (s, s) a + c with packed FMAs
__device__ __forceinline__ float2 cfma_x2(float s, float2 a, float2 c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2bits(make_float2(s, s))), "l"(f2bits(a)), "l"(f2bits(c)));
    return bitsf2(r);
}
// (s, s) a with a packed multiply
__device__ __forceinline__ float2 cscale_x2(float s, float2 a)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2bits(make_float2(s, s))), "l"(f2bits(a)));
    return bitsf2(r);
}
template <bool PK>
__device__ __forceinline__ float2 cadd_(float2 a, float2 b)
{
    if constexpr (PK) return cadd_x2(a, b);
    else return cadd(a, b);
}
template <bool PK>
__device__ __forceinline__ float2 csub_(float2 a, float2 b)
{
    if constexpr (PK) return csub_x2(a, b);
    else return csub(a, b);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 mul_i(float2 a) { return make_float2(-a.y, a.x); }
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }

// cos(2 pi j / 48), j = 0..48: every radix used here divides 48.
__host__ __device__ constexpr double cos48(int j)
{
    constexpr double t[49] = {
        1,
        0.99144486137381038,
        0.96592582628906831,
        0.92387953251128674,
        0.86602540378443871,
        0.79335334029123517,
        0.70710678118654757,
        0.60876142900872066,
        0.50000000000000011,
        0.38268343236508984,
        0.25881904510252074,
        0.13052619222005171,
        6.123233995736766e-17,
        -0.1305261922200516,
        -0.25881904510252063,
        -0.3826834323650895,
        -0.49999999999999978,
        -0.60876142900872066,
        -0.70710678118654746,
        -0.79335334029123505,
        -0.86602540378443871,
        -0.92387953251128674,
        -0.9659258262890682,
        -0.99144486137381038,
        -1,
        -0.99144486137381038,
        -0.96592582628906831,
        -0.92387953251128685,
        -0.86602540378443882,
        -0.79335334029123517,
        -0.70710678118654791,
        -0.60876142900872088,
        -0.50000000000000044,
        -0.3826834323650895,
        -0.25881904510252063,
        -0.13052619222005163,
        -1.8369701987210297e-16,
        0.13052619222005127,
        0.2588190451025203,
        0.38268343236508917,
        0.50000000000000011,
        0.60876142900871988,
        0.70710678118654735,
        0.79335334029123494,
        0.86602540378443837,
        0.92387953251128685,
        0.96592582628906809,
        0.99144486137381038,
        1};
    return t[j];
}

// Multiply by W_R^K = exp(s 2 pi i K / R), s = -1 forward, +1 inverse.
template <int R, int K, bool FWD>
__device__ __forceinline__ float2 twmul(float2 a)
{
    static_assert(48 % R == 0, "radix must divide 48");
    constexpr int j = (K * (48 / R)) % 48;
    if constexpr (j == 0) {
        return a;
    } else if constexpr (j == 12) {   // W = -i (fwd) / +i (inv)
        return FWD ? mul_mi(a) : mul_i(a);
    } else if constexpr (j == 24) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (j == 36) {
        return FWD ? mul_i(a) : mul_mi(a);
    } else {
        constexpr float c = (float)cos48(j);
        constexpr float s = (float)cos48((j + 36) % 48) * (FWD ? -1.0f : 1.0f);
        return cmul(a, make_float2(c, s));
    }
}

// In-register R-point DFT, natural order in and out; PK: packed FP32x2
// complex adds.
template <int R, bool FWD, bool PK = false>
struct Dft {
    template <int K>
    static __device__ __forceinline__ void combine(float2 *v, const float2 *e, const float2 *o)
    {
        if constexpr (K < R / 2) {
            constexpr int j = (K * (48 / R)) % 48;
            if constexpr (j % 12 == 6) {
                // W = h (sc + i ss) with h = sqrt(2)/2: o W = h (A + i B), and
                // the butterfly is four FMAs on e
                constexpr float h = 0.70710678118654752f;
                constexpr float sc = (j == 6 || j == 42) ? 1.f : -1.f;                      // sign of cos
                constexpr float ss = ((j == 6 || j == 18) ? 1.f : -1.f) * (FWD ? -1.f : 1.f);   // sign of sin
                const float A = sc * o[K].x - ss * o[K].y;
                const float B = ss * o[K].x + sc * o[K].y;
                if constexpr (PK) {
                    v[K] = cfma_x2(h, make_float2(A, B), e[K]);
                    v[K + R / 2] = cfma_x2(-h, make_float2(A, B), e[K]);
                } else {
                    v[K] = make_float2(fmaf(h, A, e[K].x), fmaf(h, B, e[K].y));
                    v[K + R / 2] = make_float2(fmaf(-h, A, e[K].x), fmaf(-h, B, e[K].y));
                }
            } else {
                const float2 t = twmul<R, K, FWD>(o[K]);
                v[K] = cadd_<PK>(e[K], t);
                v[K + R / 2] = csub_<PK>(e[K], t);
            }
            combine<K + 1>(v, e, o);
        }
    }
    static __device__ __forceinline__ void run(float2 *v)
    {
        static_assert(R % 2 == 0, "odd radix needs its own base case");
        constexpr int H = R / 2;
        float2 e[H], o[H];
#pragma unroll
        for (int i = 0; i < H; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        Dft<H, FWD, PK>::run(e);
        Dft<H, FWD, PK>::run(o);
        combine<0>(v, e, o);
    }
};

template <bool FWD, bool PK>
struct Dft<1, FWD, PK> {
    static __device__ __forceinline__ void run(float2 *) {}
};

template <bool FWD, bool PK>
struct Dft<2, FWD, PK> {
    static __device__ __forceinline__ void run(float2 *v)
    {
        const float2 a = v[0], b = v[1];
        v[0] = cadd_<PK>(a, b);
        v[1] = csub_<PK>(a, b);
    }
};

template <bool FWD, bool PK>
struct Dft<3, FWD, PK> {
    static __device__ __forceinline__ void run(float2 *v)
    {
        // X1,2 = v0 - (v1+v2)/2 -/+ s i (sqrt3/2)(v1 - v2), s = +1 fwd
        constexpr float h = 0.86602540378443865f;
        const float2 s = cadd(v[1], v[2]);
        const float2 d = cscale(csub(v[1], v[2]), FWD ? -h : h);
        const float2 m = make_float2(v[0].x - 0.5f * s.x, v[0].y - 0.5f * s.y);
        v[0] = cadd(v[0], s);
        v[1] = cadd(m, mul_i(d));
        v[2] = csub(m, mul_i(d));
    }
};

// Plans: N = R0 * R1 (* R2), P threads per line, V = N / P values per thread.
template <int N>
struct Plan;
template <> struct Plan<16>  { static constexpr int P = 4,  NP = 2, R0 = 4,  R1 = 4,  R2 = 1; };
template <> struct Plan<32>  { static constexpr int P = 4,  NP = 2, R0 = 8,  R1 = 4,  R2 = 1; };
template <> struct Plan<64>  { static constexpr int P = 8,  NP = 2, R0 = 8,  R1 = 8,  R2 = 1; };
template <> struct Plan<128> { static constexpr int P = 8,  NP = 2, R0 = 16, R1 = 8,  R2 = 1; };
template <> struct Plan<256> { static constexpr int P = 16, NP = 2, R0 = 16, R1 = 16, R2 = 1; };
template <> struct Plan<384> { static constexpr int P = 16, NP = 3, R0 = 8,  R1 = 6,  R2 = 8; };
template <> struct Plan<512> { static constexpr int P = 32, NP = 3, R0 = 8,  R1 = 8,  R2 = 8; };

// Alternative plans with more threads per line (fewer values and registers
// per thread, one more exchange), offered to the autotuner for the x passes.
// VAR 0 is Plan<N>; sizes without an alternative reuse it.
template <int N, int VAR>
struct PlanV : Plan<N> {};
template <> struct PlanV<128, 1> { static constexpr int P = 16, NP = 3, R0 = 8, R1 = 2, R2 = 8; };
template <> struct PlanV<256, 1> { static constexpr int P = 32, NP = 3, R0 = 8, R1 = 4, R2 = 8; };
template <> struct PlanV<512, 1> { static constexpr int P = 64, NP = 3, R0 = 8, R1 = 8, R2 = 8; };
__host__ __device__ constexpr bool has_plan_variant(int N) { return N == 128 || N == 256 || N == 512; }

template <int N, int VAR = 0>
struct PlanInfo {
    using PL = PlanV<N, VAR>;
    static constexpr int P = PL::P;
    static constexpr int V = N / P;
    static constexpr int NP = PL::NP;
    static constexpr int R0 = PL::R0, R1 = PL::R1, R2 = PL::R2;
    static constexpr int RL = NP == 2 ? R1 : R2;        // radix of the last pass
    static constexpr bool matched = (R0 == RL);        // last-pass positions == first-pass positions
    static_assert(R0 * R1 * R2 == N, "plan must factor N");
    static_assert(N % (R0 * P) == 0 && N % (R1 * P) == 0 && (R2 == 1 || N % (R2 * P) == 0), "plan/P mismatch");
    // position of register slot i in the first pass' input order
    static __device__ __forceinline__ int in_pos(int p, int i)
    {
        return p + (i / R0) * P + (i % R0) * (N / R0);
    }
    // position of register slot i in the last pass' output order
    static __device__ __forceinline__ int out_pos(int p, int i)
    {
        return p + (i / RL) * P + (i % RL) * (N / RL);
    }
};

// One radix-R pass on the registers: twiddles then R-point DFTs.
template <int N, int R, int Ns, int P, bool FWD, bool PK = false>
__device__ __forceinline__ void pass_regs(float2 *v, int p, const float2 *__restrict__ tw)
{
    constexpr int B = N / (R * P);
#pragma unroll
    for (int b = 0; b < B; ++b) {
        if constexpr (Ns > 1) {
            const int j = p + b * P;
            const int k = j % Ns;
#pragma unroll
            for (int t = 1; t < R; ++t) {
                float2 w = tw[t * k * (N / (Ns * R))];
                if (!FWD) w.y = -w.y;
                v[b * R + t] = cmul(v[b * R + t], w);
            }
        }
        Dft<R, FWD, PK>::run(&v[b * R]);
    }
}

// The barrier of the column-pass exchanges: the whole block, or (NamedSync)
// the ID-th hardware barrier over COUNT threads, for kernels whose warps
// form groups doing different work.
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
template <int ID, int COUNT>
struct NamedSync {
    __device__ __forceinline__ void operator()() const { asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(COUNT) : "memory"); }
};

// Hand the outputs of a pass (radix R, Ns) to the next pass (radix R2n).
// `at(pos)` returns the shared-memory slot of line position pos for this
// thread's line.  Brackets the exchange with block (or group) barriers.
template <int N, int R, int Ns, int Rn, int P, class At, class Sync = BlockSync>
__device__ __forceinline__ void exchange(float2 *v, int p, At at, Sync sync = Sync())
{
    constexpr int B = N / (R * P);
    constexpr int Bn = N / (Rn * P);
    sync();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = p + b * P;
        const int base = (j / Ns) * Ns * R + (j % Ns);
#pragma unroll
        for (int t = 0; t < R; ++t) *at(base + t * Ns) = v[b * R + t];
    }
    sync();
#pragma unroll
    for (int b = 0; b < Bn; ++b) {
        const int j = p + b * P;
#pragma unroll
        for (int t = 0; t < Rn; ++t) v[b * Rn + t] = *at(j + t * (N / Rn));
    }
}

// Full line transform.  In: v in first-pass input order.  Out: v in
// last-pass output order (PlanInfo::out_pos).  Every thread of the block (of
// the group, with a NamedSync) must call it: it contains barriers.
template <int N, bool FWD, int VAR = 0, class At, class Sync = BlockSync>
__device__ __forceinline__ void fft_line(float2 *v, int p, const float2 *__restrict__ tw, At at, Sync sync = Sync())
{
    using PI = PlanInfo<N, VAR>;
    constexpr int P = PI::P;
    pass_regs<N, PI::R0, 1, P, FWD>(v, p, tw);
    exchange<N, PI::R0, 1, PI::R1, P>(v, p, at, sync);
    pass_regs<N, PI::R1, PI::R0, P, FWD>(v, p, tw);
    if constexpr (PI::NP == 3) {
        exchange<N, PI::R1, PI::R0, PI::R2, P>(v, p, at, sync);
        pass_regs<N, PI::R2, PI::R0 * PI::R1, P, FWD>(v, p, tw);
    }
}

// ---------------------------------------------------------------------------
// Warp-local lines: a line lives inside one warp (P <= 32 threads, 32/P
// lines per warp), so the pass exchanges need only __syncwarp and warps run
// independently of each other.  Used by the contiguous-axis (z) passes.
// ---------------------------------------------------------------------------
template <int N>
struct WPlan;
template <> struct WPlan<16>  { static constexpr int P = 4,  NP = 2, R0 = 4,  R1 = 4, R2 = 1, R3 = 1; };
template <> struct WPlan<32>  { static constexpr int P = 8,  NP = 3, R0 = 4,  R1 = 2, R2 = 4, R3 = 1; };
template <> struct WPlan<64>  { static constexpr int P = 8,  NP = 2, R0 = 8,  R1 = 8, R2 = 1, R3 = 1; };
template <> struct WPlan<128> { static constexpr int P = 16, NP = 3, R0 = 8,  R1 = 2, R2 = 8, R3 = 1; };
template <> struct WPlan<256> { static constexpr int P = 32, NP = 3, R0 = 8,  R1 = 4, R2 = 8, R3 = 1; };
template <> struct WPlan<384> { static constexpr int P = 32, NP = 4, R0 = 4,  R1 = 4, R2 = 6, R3 = 4; };
template <> struct WPlan<512> { static constexpr int P = 32, NP = 3, R0 = 16, R1 = 2, R2 = 16, R3 = 1; };

// Alternative warp-local plans offered to the autotuner for the z pass:
// VAR 1 at N = 256 is a two-pass 16 x 16 plan on 16 threads per line (one
// exchange per line transform instead of two; twice the values per thread).
template <int N, int VAR>
struct WPlanV : WPlan<N> {};
template <> struct WPlanV<256, 1> { static constexpr int P = 16, NP = 2, R0 = 16, R1 = 16, R2 = 1, R3 = 1; };
__host__ __device__ constexpr bool has_zplan_variant(int N) { return N == 256; }

template <int N, int VAR = 0>
struct WPlanInfo {
    using PL = WPlanV<N, VAR>;
    static constexpr int P = PL::P;
    static constexpr int V = N / P;
    static constexpr int NP = PL::NP;
    static constexpr int R0 = PL::R0, R1 = PL::R1, R2 = PL::R2, R3 = PL::R3;
    static constexpr int RL = NP == 2 ? R1 : (NP == 3 ? R2 : R3);
    static constexpr bool matched = (R0 == RL);
    static_assert(R0 * R1 * R2 * R3 == N, "plan must factor N");
    static_assert(32 % P == 0, "a line must fit in one warp");
    static_assert(V % R0 == 0 && V % R1 == 0 && V % R2 == 0 && V % R3 == 0, "radix must divide V");
    static __device__ __forceinline__ int in_pos(int p, int i) { return p + (i / R0) * P + (i % R0) * (N / R0); }
    static __device__ __forceinline__ int out_pos(int p, int i) { return p + (i / RL) * P + (i % RL) * (N / RL); }
};

template <int N, int R, int Ns, int Rn, int P, class At>
__device__ __forceinline__ void exchange_warp(float2 *v, int p, At at)
{
    constexpr int B = N / (R * P);
    constexpr int Bn = N / (Rn * P);
    __syncwarp();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = p + b * P;
        const int base = (j / Ns) * Ns * R + (j % Ns);
#pragma unroll
        for (int t = 0; t < R; ++t) *at(base + t * Ns) = v[b * R + t];
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < Bn; ++b) {
        const int j = p + b * P;
#pragma unroll
        for (int t = 0; t < Rn; ++t) v[b * Rn + t] = *at(j + t * (N / Rn));
    }
}

// Per-thread inter-pass twiddles of a warp-local plan, held in registers.
// Pass s (radix R, after Ns points) multiplies slot t of butterfly b by
// W_N^{t k N/(Ns R)}, k = (p + b P) mod Ns; the forward values are stored,
// the inverse uses their conjugates.
template <int N, int R, int Ns, int P>
struct PassTw {
    static constexpr int B = N / (R * P);
    float2 w[B][R > 1 ? R - 1 : 1];
    __device__ __forceinline__ void init(int p, const float2 *__restrict__ tw)
    {
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int k = (p + b * P) % Ns;
#pragma unroll
            for (int t = 1; t < R; ++t) w[b][t - 1] = tw[t * k * (N / (Ns * R))];
        }
    }
};

template <int N, int R, int Ns, int P, bool FWD, bool PK = false>
__device__ __forceinline__ void pass_regs_tw(float2 *v, const PassTw<N, R, Ns, P> &T)
{
    constexpr int B = N / (R * P);
#pragma unroll
    for (int b = 0; b < B; ++b) {
#pragma unroll
        for (int t = 1; t < R; ++t) {
            float2 w = T.w[b][t - 1];
            if (!FWD) w.y = -w.y;
            v[b * R + t] = cmul(v[b * R + t], w);
        }
        Dft<R, FWD, PK>::run(&v[b * R]);
    }
}

template <int N, int VAR = 0>
struct WarpTw {
    using PI = WPlanInfo<N, VAR>;
    static constexpr int P = PI::P, R0 = PI::R0, R1 = PI::R1, R2 = PI::R2, R3 = PI::R3;
    PassTw<N, R1, R0, P> t1;
    PassTw<N, (PI::NP >= 3 ? R2 : 2), R0 * R1, P> t2;
    PassTw<N, (PI::NP >= 4 ? R3 : 2), R0 * R1 * R2, P> t3;
    __device__ __forceinline__ void init(int p, const float2 *__restrict__ tw)
    {
        t1.init(p, tw);
        if constexpr (PI::NP >= 3) t2.init(p, tw);
        if constexpr (PI::NP >= 4) t3.init(p, tw);
    }
};

// Padded exchange layouts of the power-of-two warp-local plans (WPlan<N>).
// Exchange s (after pass s) puts line position pos at slot
// pos + (pos >> A_s) * D_s of the line's shared row.  Every position an
// exchange touches is a per-lane part plus a compile-time part (butterfly
// index, radix slot) with disjoint bits, and the map is additive over such
// parts, so each access is one per-lane base plus an immediate offset: no
// per-access address arithmetic.  A_s, D_s and the row stride SROW are the
// bank-conflict-free choices printed by tests/swizzle_search.py (half-warp model
// of 8-byte requests).
template <int N>
struct WPad {
    static constexpr bool on = false;
    static constexpr int SROW = 0, A0 = 0, D0 = 0, A1 = 0, D1 = 0;
};
template <> struct WPad<16>  { static constexpr bool on = true; static constexpr int SROW = 20,  A0 = 2, D0 = 1, A1 = 0, D1 = 0; };
template <> struct WPad<32>  { static constexpr bool on = true; static constexpr int SROW = 40,  A0 = 3, D0 = 1, A1 = 1, D1 = 0; };
template <> struct WPad<64>  { static constexpr bool on = true; static constexpr int SROW = 72,  A0 = 3, D0 = 1, A1 = 0, D1 = 0; };
template <> struct WPad<128> { static constexpr bool on = true; static constexpr int SROW = 184, A0 = 4, D0 = 1, A1 = 4, D1 = 8; };
template <> struct WPad<256> { static constexpr bool on = true; static constexpr int SROW = 312, A0 = 4, D0 = 1, A1 = 5, D1 = 8; };
template <> struct WPad<512> { static constexpr bool on = true; static constexpr int SROW = 543, A0 = 4, D0 = 1, A1 = 1, D1 = 0; };

// the same per plan variant (WPlanV<N, VAR>): VAR 0 is WPad<N>
template <int N, int VAR>
struct WPadV {
    static constexpr bool on = false;
    static constexpr int SROW = 0, A0 = 0, D0 = 0, A1 = 0, D1 = 0;
};
template <int N> struct WPadV<N, 0> : WPad<N> {};
template <> struct WPadV<256, 1> { static constexpr bool on = true; static constexpr int SROW = 271, A0 = 4, D0 = 1, A1 = 0, D1 = 0; };

template <int A, int D>
__host__ __device__ constexpr int pad_slot(int x)
{
    return x + (x >> A) * D;
}

template <int N, int R, int Ns, int Rn, int P, int A, int D>
__device__ __forceinline__ void exchange_warp_pad(float2 *v, int p, float2 *row)
{
    static_assert(P % Ns == 0 || Ns % P == 0, "lane and butterfly parts of a position must not overlap");
    constexpr int B = N / (R * P);
    constexpr int Bn = N / (Rn * P);
    // store: position (j / Ns) Ns R + (j mod Ns) + t Ns, j = p + b P
    float2 *st = row + pad_slot<A, D>(P % Ns == 0 ? (p / Ns) * Ns * R + p % Ns : p);
    __syncwarp();
#pragma unroll
    for (int b = 0; b < B; ++b) {
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int c = P % Ns == 0 ? b * P * R + t * Ns : (b * P / Ns) * Ns * R + (b * P) % Ns + t * Ns;
            st[pad_slot<A, D>(c)] = v[b * R + t];
        }
    }
    __syncwarp();
    // load: position p + b P + t N / Rn
    const float2 *ld = row + pad_slot<A, D>(p);
#pragma unroll
    for (int b = 0; b < Bn; ++b) {
#pragma unroll
        for (int t = 0; t < Rn; ++t) v[b * Rn + t] = ld[pad_slot<A, D>(b * P + t * (N / Rn))];
    }
}

// Inter-pass twiddles of a warp plan in shared memory, lane-major: entry
// (pass s, butterfly b, slot t) of lane p at [offset_s + (b (R - 1) + t - 1)
// P + p], the value WarpTw holds in registers.  A warp's request for one
// (s, b, t) reads P consecutive entries: no bank conflicts.  Fewer registers
// are held across the transforms than with WarpTw.
template <int N>
struct LaneTw {
    using PI = WPlanInfo<N, 0>;
    static constexpr int P = PI::P, R0 = PI::R0, R1 = PI::R1, R2 = PI::R2;
    static constexpr int B1 = N / (R1 * P), B2 = PI::NP >= 3 ? N / (R2 * P) : 0;
    static constexpr int OFF2 = B1 * (R1 - 1) * P;
    static constexpr int SIZE = OFF2 + (PI::NP >= 3 ? B2 * (R2 - 1) * P : 0);   // float2
    // whole block; tw: the N-entry table W_N^m
    static __device__ __forceinline__ void init(float2 *tab, const float2 *tw)
    {
        for (int i = threadIdx.x; i < SIZE; i += blockDim.x) {
            const bool second = i >= OFF2;
            const int j = second ? i - OFF2 : i;
            const int R = second ? R2 : R1, Ns = second ? R0 * R1 : R0;
            const int p = j % P, bt = j / P, b = bt / (R - 1), t = bt % (R - 1) + 1;
            const int k = (p + b * P) % Ns;
            tab[i] = tw[t * k * (N / (Ns * R))];
        }
    }
};

template <int N, int R, int Ns, int P, bool FWD, bool PK>
__device__ __forceinline__ void pass_regs_lt(float2 *v, const float2 *__restrict__ lt)
{
    constexpr int B = N / (R * P);
#pragma unroll
    for (int b = 0; b < B; ++b) {
#pragma unroll
        for (int t = 1; t < R; ++t) {
            float2 w = lt[(b * (R - 1) + t - 1) * P];
            if (!FWD) w.y = -w.y;
            v[b * R + t] = cmul(v[b * R + t], w);
        }
        Dft<R, FWD, PK>::run(&v[b * R]);
    }
}

// Line transform of the default warp plan through the padded layouts with
// the lane-major shared twiddles (tab: LaneTw<N> table).
template <int N, bool FWD>
__device__ __forceinline__ void fft_line_warp_pad_lt(float2 *v, int p, const float2 *__restrict__ tab, float2 *row)
{
    using PI = WPlanInfo<N, 0>;
    using PD = WPadV<N, 0>;
    using LT = LaneTw<N>;
    static_assert(PD::on && PI::NP <= 3, "padded layouts exist for the power-of-two plans");
    constexpr int P = PI::P, R0 = PI::R0, R1 = PI::R1, R2 = PI::R2;
    pass_regs<N, R0, 1, P, FWD, true>(v, p, nullptr);
    exchange_warp_pad<N, R0, 1, R1, P, PD::A0, PD::D0>(v, p, row);
    pass_regs_lt<N, R1, R0, P, FWD, true>(v, tab + p);
    if constexpr (PI::NP == 3) {
        exchange_warp_pad<N, R1, R0, R2, P, PD::A1, PD::D1>(v, p, row);
        pass_regs_lt<N, R2, R0 * R1, P, FWD, true>(v, tab + LT::OFF2 + p);
    }
}

// Line transform of a warp plan through the padded layouts; row is this
// line's shared row (WPadV<N, VAR>::SROW slots).
template <int N, bool FWD, int VAR = 0>
__device__ __forceinline__ void fft_line_warp_pad(float2 *v, int p, const WarpTw<N, VAR> &T, float2 *row)
{
    using PI = WPlanInfo<N, VAR>;
    using PD = WPadV<N, VAR>;
    static_assert(PD::on && PI::NP <= 3, "padded layouts exist for the power-of-two plans");
    constexpr int P = PI::P, R0 = PI::R0, R1 = PI::R1, R2 = PI::R2;
    pass_regs<N, R0, 1, P, FWD, true>(v, p, nullptr);
    exchange_warp_pad<N, R0, 1, R1, P, PD::A0, PD::D0>(v, p, row);
    pass_regs_tw<N, R1, R0, P, FWD, true>(v, T.t1);
    if constexpr (PI::NP == 3) {
        exchange_warp_pad<N, R1, R0, R2, P, PD::A1, PD::D1>(v, p, row);
        pass_regs_tw<N, R2, R0 * R1, P, FWD, true>(v, T.t2);
    }
}

// Warp-local line transform with register twiddles.
template <int N, bool FWD, int VAR = 0, class At>
__device__ __forceinline__ void fft_line_warp_tw(float2 *v, int p, const WarpTw<N, VAR> &T, At at)
{
    using PI = WPlanInfo<N, VAR>;
    constexpr int P = PI::P;
    constexpr int R0 = PI::R0, R1 = PI::R1, R2 = PI::R2, R3 = PI::R3;
    pass_regs<N, R0, 1, P, FWD, true>(v, p, nullptr);
    exchange_warp<N, R0, 1, R1, P>(v, p, at);
    pass_regs_tw<N, R1, R0, P, FWD, true>(v, T.t1);
    if constexpr (PI::NP >= 3) {
        exchange_warp<N, R1, R0, R2, P>(v, p, at);
        pass_regs_tw<N, R2, R0 * R1, P, FWD, true>(v, T.t2);
    }
    if constexpr (PI::NP >= 4) {
        exchange_warp<N, R2, R0 * R1, R3, P>(v, p, at);
        pass_regs_tw<N, R3, R0 * R1 * R2, P, FWD, true>(v, T.t3);
    }
}

// Warp-local line transform; all 32 lanes of the warp must call it.
template <int N, bool FWD, class At>
__device__ __forceinline__ void fft_line_warp(float2 *v, int p, const float2 *__restrict__ tw, At at)
{
    using PI = WPlanInfo<N>;
    constexpr int P = PI::P;
    constexpr int R0 = PI::R0, R1 = PI::R1, R2 = PI::R2, R3 = PI::R3;
    pass_regs<N, R0, 1, P, FWD, true>(v, p, tw);
    exchange_warp<N, R0, 1, R1, P>(v, p, at);
    pass_regs<N, R1, R0, P, FWD, true>(v, p, tw);
    if constexpr (PI::NP >= 3) {
        exchange_warp<N, R1, R0, R2, P>(v, p, at);
        pass_regs<N, R2, R0 * R1, P, FWD, true>(v, p, tw);
    }
    if constexpr (PI::NP >= 4) {
        exchange_warp<N, R2, R0 * R1, R3, P>(v, p, at);
        pass_regs<N, R3, R0 * R1 * R2, P, FWD, true>(v, p, tw);
    }
}

}  // namespace ens
