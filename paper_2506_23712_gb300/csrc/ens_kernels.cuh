// Hot-path kernels of the ensemble DNS (sm_103a).
//
// One member is a forced periodic-box Navier-Stokes DNS whose injection
// rate is exp(lambda) eps_bar (Sec. II, Eq. ensemble_hypothesis; Sec. IV).
// Its state is the dealiased half spectrum in a compact layout that stores
// only the modes the cubic 2/3 rule keeps (|k_i| <= kc = ceil(N/3) - 1), so
// every transform is pruned: the inverse passes skip the zero band and the
// forward passes drop it on output.  One RK stage is five passes:
//
//   IX  : state (3 comps) -> u, omega = i k x u, transformed along x   [A]
//   IY  : A -> transformed along y                                      [B]
//   ZNL : B -> along z to physical space, n = u x omega, max|u|, and
//         straight back along z (two real rows per complex line)        [B]
//   FY  : B -> forward along y, dealiased rows dropped                  [A]
//   FXU : A -> forward along x, 1/N^3, Leray projection, constant-power
//         band forcing, integrating-factor RK stage, FP64 partial sums  [U/S]
//
// The statistics snapshot reuses IX/IY with the eight independent gradient
// components and ends in ZSTAT: Q, R, dissipation and enstrophy per point,
// shared-memory histograms and moment sums (Secs. V-VII).
#pragma once

#include "ens_fft.cuh"
#include "ens_internal.h"

namespace ens {

// Geometry of a grid size, known at compile time (the host's Geo carries the
// same values: kc = ceil(N/3) - 1, NK = 2 kc + 1, NZ = kc + 1, NZp = NZ
// rounded up to kTile), so index arithmetic folds into constants.
template <int N>
struct Dims {
    static constexpr int KC = (N + 2) / 3 - 1;
    static constexpr int NK = 2 * KC + 1;
    static constexpr int NZ = KC + 1;
    static constexpr int NZP = (NZ + kTile - 1) / kTile * kTile;
    static constexpr long long SU = (long long)NK * NK * NZP;   // per state component
    static constexpr long long SA = (long long)NK * N * NZP;    // per buffer-A field
    static constexpr long long SB = (long long)N * N * NZP;     // per buffer-B field
};

// Shared-memory slot of position pos of a warp-local line.  For the large
// sizes an XOR swizzle permutes the 16 slots of every 16-aligned block by a
// 4-bit mask of that block (table packed into two 64-bit words), chosen by an
// offline search over every access pattern of the line transforms (the pass
// exchanges, the output stores, the Hermitian unpacking reads) so that each
// half-warp request of 8-byte words meets 16 distinct bank pairs
// (tests/swizzle_search.py reproduces the tables); the
// small sizes keep an additive padding.
template <int N>
struct RowSwz {
    static constexpr bool on = false;
    static constexpr unsigned long long lo = 0, hi = 0;
};
template <> struct RowSwz<128> { static constexpr bool on = true; static constexpr unsigned long long lo = 0x7ed43a90ull, hi = 0; };
template <> struct RowSwz<256> { static constexpr bool on = true; static constexpr unsigned long long lo = 0x01ab45effe54ba10ull, hi = 0; };
template <> struct RowSwz<384> { static constexpr bool on = true; static constexpr unsigned long long lo = 0xf906c1a7af41872dull, hi = 0xd42bc2b5ull; };
template <> struct RowSwz<512> { static constexpr bool on = true; static constexpr unsigned long long lo = 0xf01695843ea7bd2cull, hi = 0xcc22bb3311504988ull; };

// rows handled per CTA by the z-direction passes
template <int N>
struct RowCfg {
    static constexpr int P = WPlanInfo<N>::P;     // threads per row (warp-local lines)
    static constexpr int RZ = 256 / P;            // rows per 256-thread CTA
    // shared row stride (float2): swizzled rows are dense, padded rows are not
    static constexpr int SROW = RowSwz<N>::on ? N : N + N / 16 + N / 32 + 1;
};

// Column-tile passes (x and y) take the tile width T (columns per CTA, a
// divisor of kTile) as a template parameter: the autotuner picks it per grid
// size.  Registers per thread stay the same for every T (128 at most where
// the T = kTile variant asks for two CTAs per SM).
template <int N, int T, int VAR = 0>
struct ColCfg {
    static_assert(kTile % T == 0, "tile width must divide the column padding");
    static constexpr int threads = T * PlanInfo<N, VAR>::P;
    // VAR 0 keeps 128 registers per thread where two 256-thread CTAs fit an
    // SM; the wider plans (VAR 1) aim at 1024 resident threads (<= 64 registers)
    static constexpr int min_blocks =
        VAR == 0 ? (256 / (kTile * PlanInfo<N>::P) > 0 ? 2 : 1) * (kTile / T) : (1024 / threads > 0 ? 1024 / threads : 1);
};

// Launch helpers (host): shared memory bytes per pass.
template <int N, int T>
constexpr size_t smem_cols() { return sizeof(float2) * (size_t)(N + N * T); }
__host__ __device__ constexpr int kc_of_n(int N) { return (N + 2) / 3 - 1; }
// x passes also stage the three components of a column tile: [3][NK][T]
template <int N, int T>
constexpr size_t smem_x() { return smem_cols<N, T>() + sizeof(float2) * 3 * (2 * kc_of_n(N) + 1) * T; }
template <int N>
constexpr size_t smem_rows() { return sizeof(float2) * (size_t)(N + RowCfg<N>::RZ * RowCfg<N>::SROW); }

__device__ __forceinline__ int wnum(int pos, int N) { return pos <= N / 2 ? pos : pos - N; }

// 16-byte asynchronous global -> shared copy (cp.async, L2 only); bytes < 16
// of the source are read and the rest of the destination is zero-filled
__device__ __forceinline__ void cp_async_16(void *dst, const void *src, int bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// wait until at most `Pending` of this thread's committed groups are in flight
template <int Pending>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(Pending) : "memory");
}

__device__ __forceinline__ void load_twiddles(float2 *tw, const float2 *__restrict__ g, int N)
{
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = g[i];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// IX: inverse transform along x of fields built from the state.
//   MODE 0: u_x, u_y, u_z, omega_x, omega_y, omega_z   (omega = i k x u)
//   MODE 1: A_ij = i k_j u_i for ij = 11,12,13,21,22,23,31,32
// grid (NK*NZp/T, members), block T*P.
// ---------------------------------------------------------------------------
// The pass bodies take their block coordinates (column tile bx, field,
// member m) and shared memory as arguments: the __global__ kernels pass
// blockIdx and their dynamic shared memory, the persistent stage kernel
// (ens_persist.cu) the coordinates of the work item it runs.
template <int N, int MODE, int T, int VAR = 0>
__device__ __forceinline__ void inv_x_body(const Geo &g, int use_S, int bx, int m, float2 *sm)
{
    using PI = PlanInfo<N, VAR>;
    constexpr int P = PI::P, V = PI::V;
    float2 *tw = sm, *buf = sm + N, *tile = buf + N * T;   // tile: [3][NK][T]

    const int c = threadIdx.x % T, p = threadIdx.x / T;
    const int col0 = bx * T;                            // a tile never straddles ky (NZp % T == 0)
    const int col = col0 + c;
    const int iy = col / Dims<N>::NZP, kz = col % Dims<N>::NZP;
    const int kz0 = col0 % Dims<N>::NZP;                  // first kz of the tile
    const bool valid = kz < Dims<N>::NZ;
    const float ky = (float)(iy <= Dims<N>::KC ? iy : iy - Dims<N>::NK);
    const float kzf = (float)kz;
    const long long rowU = (long long)Dims<N>::NK * Dims<N>::NZP;
    const float2 *X = (use_S ? g.S : g.U) + (long long)m * 3 * Dims<N>::SU + col0;
    // staging of the three velocity components of this column tile with
    // asynchronous 16-byte copies (two columns each, the dealiased columns
    // zero-filled), one commit group per component in the order the
    // transforms use them: the whole tile is in flight at once, no registers
    // held, and the first transform starts once its component has landed
    constexpr int per = Dims<N>::NK * T;
    constexpr int order[3] = {MODE == 0 ? 1 : 0, MODE == 0 ? 2 : 1, MODE == 0 ? 0 : 2};
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const int q = order[s];
        for (int idx = 2 * threadIdx.x; idx < per; idx += 2 * blockDim.x) {
            const int ix = idx / T, cc = idx % T;   // cc even
            const int nvalid = min(max(Dims<N>::NZ - (kz0 + cc), 0), 2);
            cp_async_16(&tile[q * per + idx], X + q * Dims<N>::SU + ix * rowU + cc, 8 * nvalid);
        }
        cp_async_commit();
    }
    load_twiddles(tw, g.tw, N);
    // component order[s] complete and visible to the block
    auto landed = [&](int s) {
        if (s == 0) cp_async_wait<2>();
        else if (s == 1) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncthreads();
    };

    float2 *dst0 = g.A + (long long)m * kFields * Dims<N>::SA + ((long long)iy * N) * Dims<N>::NZP + kz;
    auto at = [&](int pos) { return &buf[pos * T + c]; };
    // transform of component q of the tile, optionally times i kx (the x
    // derivative: kx varies along this transform, so it is applied before it)
    auto transform = [&](float2 *v, int q, bool dx) {
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const int kxi = wnum(PI::in_pos(p, i), N);
            const bool keep = kxi >= -Dims<N>::KC && kxi <= Dims<N>::KC;
            const int ix = kxi >= 0 ? kxi : kxi + Dims<N>::NK;
            const float2 u = keep ? tile[q * per + ix * T + c] : make_float2(0.f, 0.f);
            v[i] = dx ? mul_i(cscale(u, (float)kxi)) : u;
        }
        fft_line<N, false, VAR>(v, p, tw, at);
    };
    auto store = [&](const float2 *v, int f) {
        if (valid) {
            float2 *dst = dst0 + (long long)f * Dims<N>::SA;
#pragma unroll
            for (int i = 0; i < V; ++i) dst[(long long)PI::out_pos(p, i) * Dims<N>::NZP] = v[i];
        }
    };
    // ky and kz are constant along x, so their derivatives are applied after
    // the transform: 5 transforms give u and omega; for the gradient the 6
    // transforms of u_i and i kx u_i go to the y pass, which applies ky, kz
    float2 Ua[V], Ub[V];
    if constexpr (MODE == 0) {
        // omega = i k x u: (k x u)_x = ky uz - kz uy, _y = kz ux - kx uz, _z = kx uy - ky ux
        landed(0);
        transform(Ua, 1, false);                                  // uy
        store(Ua, 1);
        landed(1);
        transform(Ub, 2, false);                                  // uz
        store(Ub, 2);
#pragma unroll
        for (int i = 0; i < V; ++i)
            Ua[i] = mul_i(make_float2(ky * Ub[i].x - kzf * Ua[i].x, ky * Ub[i].y - kzf * Ua[i].y));
        store(Ua, 3);                                             // omega_x
        landed(2);
        transform(Ua, 0, false);                                  // ux
        store(Ua, 0);
        transform(Ub, 2, true);                                   // i kx uz
#pragma unroll
        for (int i = 0; i < V; ++i)
            Ub[i] = make_float2(-kzf * Ua[i].y - Ub[i].x, kzf * Ua[i].x - Ub[i].y);   // i kz ux - i kx uz
        store(Ub, 4);                                             // omega_y
        transform(Ub, 1, true);                                   // i kx uy
#pragma unroll
        for (int i = 0; i < V; ++i)
            Ub[i] = make_float2(Ub[i].x + ky * Ua[i].y, Ub[i].y - ky * Ua[i].x);      // i kx uy - i ky ux
        store(Ub, 5);                                             // omega_z
    } else {
        // velocity gradient A_ij = i k_j u_i, x part: u_i to field i and
        // i kx u_i to field 3 + i; the y pass forms the ky and kz
        // derivatives from field i (k_inv_y_grad)
#pragma unroll 1
        for (int ci = 0; ci < 3; ++ci) {
            landed(ci);
            transform(Ua, ci, false);
            store(Ua, ci);
            transform(Ub, ci, true);
            store(Ub, 3 + ci);
        }
    }
}

template <int N, int MODE, int T, int VAR = 0>
__global__ void __launch_bounds__(ColCfg<N, T, VAR>::threads, ColCfg<N, T, VAR>::min_blocks)
k_inv_x(Geo g, int use_S)
{
    extern __shared__ __align__(16) float2 sm[];
    inv_x_body<N, MODE, T, VAR>(g, use_S, blockIdx.x, blockIdx.y, sm);
}

// ---------------------------------------------------------------------------
// IY: inverse transform along y of buffer-A fields [f0, f0+nf) into B.
// grid (N*NZp/T, nf, members).
// ---------------------------------------------------------------------------
template <int N, int T, int VAR = 0>
__device__ __forceinline__ void inv_y_body(const Geo &g, int bx, int f, int m, float2 *sm)
{
    using PI = PlanInfo<N, VAR>;
    constexpr int P = PI::P, V = PI::V;
    float2 *tw = sm, *buf = sm + N;
    load_twiddles(tw, g.tw, N);
    const int c = threadIdx.x % T, p = threadIdx.x / T;
    const int col = bx * T + c;               // (x, kz) flat
    const bool valid = (col % Dims<N>::NZP) < Dims<N>::NZ;
    const long long row = (long long)N * Dims<N>::NZP;
    const float2 *src = g.A + ((long long)m * kFields + f) * Dims<N>::SA + col;
    float2 *dst = g.B + ((long long)m * kFields + f) * Dims<N>::SB + col;
    float2 v[V];
#pragma unroll
    for (int i = 0; i < V; ++i) {
        const int ky = wnum(PI::in_pos(p, i), N);
        const bool keep = valid && ky >= -Dims<N>::KC && ky <= Dims<N>::KC;
        const int iy = ky >= 0 ? ky : ky + Dims<N>::NK;
        v[i] = keep ? src[iy * row] : make_float2(0.f, 0.f);
    }
    fft_line<N, false, VAR>(v, p, tw, [&](int pos) { return &buf[pos * T + c]; });
    if (valid) {
#pragma unroll
        for (int i = 0; i < V; ++i) dst[PI::out_pos(p, i) * row] = v[i];
    }
}

template <int N, int T, int VAR = 0>
__global__ void __launch_bounds__(ColCfg<N, T, VAR>::threads)
k_inv_y(Geo g, int f0)
{
    extern __shared__ __align__(16) float2 sm[];
    inv_y_body<N, T, VAR>(g, blockIdx.x, f0 + blockIdx.y, blockIdx.z, sm);
}

// IY of the velocity gradient (statistics snapshot): from the six x-pass
// fields of a member (u_i in field i, i kx u_i in field 3 + i) the eight
// stored components A_ij = i k_j u_i into B field 3 i + j (A_33 = -A_11 -
// A_22 is not stored):
//   j = 1 : transform of field 3 + i
//   j = 2 : transform of i ky times field i (ky varies along y: applied
//           before the transform)
//   j = 3 : i kz times the transform of field i (kz is constant along y:
//           applied after it), i < 2
// so the x pass writes and this pass reads six fields instead of eight.  One
// transform per CTA; the eight jobs of a column tile are consecutive CTAs
// (blockIdx.x), so the second read of field i comes from L2.
// grid (8, N*NZp/T, members).
// (N <= 256: registers capped for 40 resident warps per SM, the plain y
// pass's occupancy; the larger plans keep their registers)
template <int N, int T>
__global__ void __launch_bounds__(ColCfg<N, T, 0>::threads,
                                   N <= 256 ? (1280 / ColCfg<N, T, 0>::threads < 32 ? 1280 / ColCfg<N, T, 0>::threads : 32) : 1)
k_inv_y_grad(Geo g)
{
    using PI = PlanInfo<N, 0>;
    constexpr int P = PI::P, V = PI::V;
    extern __shared__ __align__(16) float2 sm[];
    float2 *tw = sm, *buf = sm + N;
    load_twiddles(tw, g.tw, N);
    const int fo = blockIdx.x, m = blockIdx.z;
    const int ci = fo / 3, jj = fo % 3;
    const int fi = jj == 0 ? 3 + ci : ci;
    const int c = threadIdx.x % T, p = threadIdx.x / T;
    const int col = blockIdx.y * T + c;        // (x, kz) flat
    const int kz = col % Dims<N>::NZP;
    const bool valid = kz < Dims<N>::NZ;
    const long long row = (long long)N * Dims<N>::NZP;
    const float2 *src = g.A + ((long long)m * kFields + fi) * Dims<N>::SA + col;
    float2 v[V];
#pragma unroll
    for (int i = 0; i < V; ++i) {
        const int ky = wnum(PI::in_pos(p, i), N);
        const bool keep = valid && ky >= -Dims<N>::KC && ky <= Dims<N>::KC;
        const int iy = ky >= 0 ? ky : ky + Dims<N>::NK;
        const float2 u = keep ? src[iy * row] : make_float2(0.f, 0.f);
        v[i] = jj == 1 ? mul_i(cscale(u, (float)ky)) : u;
    }
    fft_line<N, false, 0>(v, p, tw, [&](int pos) { return &buf[pos * T + c]; });
    if (jj == 2) {
        const float kzf = (float)kz;
#pragma unroll
        for (int i = 0; i < V; ++i) v[i] = mul_i(cscale(v[i], kzf));
    }
    if (valid) {
        float2 *dst = g.B + ((long long)m * kFields + fo) * Dims<N>::SB + col;
#pragma unroll
        for (int i = 0; i < V; ++i) dst[PI::out_pos(p, i) * row] = v[i];
    }
}

// ---------------------------------------------------------------------------
// FY: forward transform along y of B fields [0, nf) into A (kept ky only).
// grid (N*NZp/T, nf, members).
// ---------------------------------------------------------------------------
template <int N, int T, int VAR = 0>
__device__ __forceinline__ void fwd_y_body(const Geo &g, int bx, int f, int m, float2 *sm)
{
    using PI = PlanInfo<N, VAR>;
    constexpr int P = PI::P, V = PI::V;
    float2 *tw = sm, *buf = sm + N;
    load_twiddles(tw, g.tw, N);
    const int c = threadIdx.x % T, p = threadIdx.x / T;
    const int col = bx * T + c;
    const bool valid = (col % Dims<N>::NZP) < Dims<N>::NZ;
    const long long row = (long long)N * Dims<N>::NZP;
    const float2 *src = g.B + ((long long)m * kFields + f) * Dims<N>::SB + col;
    float2 *dst = g.A + ((long long)m * kFields + f) * Dims<N>::SA + col;
    float2 v[V];
#pragma unroll
    for (int i = 0; i < V; ++i) v[i] = valid ? src[PI::in_pos(p, i) * row] : make_float2(0.f, 0.f);
    fft_line<N, true, VAR>(v, p, tw, [&](int pos) { return &buf[pos * T + c]; });
    if (valid) {
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const int ky = wnum(PI::out_pos(p, i), N);
            if (ky >= -Dims<N>::KC && ky <= Dims<N>::KC) dst[(ky >= 0 ? ky : ky + Dims<N>::NK) * row] = v[i];
        }
    }
}

template <int N, int T, int VAR = 0>
__global__ void __launch_bounds__(ColCfg<N, T, VAR>::threads)
k_fwd_y(Geo g)
{
    extern __shared__ __align__(16) float2 sm[];
    fwd_y_body<N, T, VAR>(g, blockIdx.x, blockIdx.y, blockIdx.z, sm);
}

// ---------------------------------------------------------------------------
// z-direction passes.  Each line is one (y, x) row of NZ complex values; two
// real rows travel as the real and imaginary parts of one complex line.
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ float2 *row_slot(float2 *buf, int r, int pos)
{
    using SW = RowSwz<N>;
    if constexpr (SW::on) {
        const int blk = pos >> 4;
        const unsigned long long w = (N <= 256 || blk < 16) ? SW::lo : SW::hi;
        return &buf[r * RowCfg<N>::SROW + (pos ^ (int)((w >> ((blk & 15) * 4)) & 15ull))];
    }
    // small sizes: one pad per 16 slots (two-pass plans), one more per 32
    // (three-pass plans)
    if constexpr (WPlanInfo<N>::NP == 2) return &buf[r * RowCfg<N>::SROW + pos + (pos >> 4)];
    else return &buf[r * RowCfg<N>::SROW + pos + (pos >> 4) + (pos >> 5)];
}

// Hermitian-extended pair line a + i b at position pos from half spectra.
__device__ __forceinline__ float2 pair_at(const float2 *__restrict__ Xa, const float2 *__restrict__ Xb,
                                          int pos, int N, int kc)
{
    if (pos == 0) {
        const float2 a = Xa[0], b = Xb[0];
        return make_float2(a.x, b.x);   // real parts only (C2R convention)
    }
    if (pos <= kc) {
        const float2 a = Xa[pos], b = Xb[pos];
        return make_float2(a.x - b.y, a.y + b.x);
    }
    if (pos >= N - kc) {
        const float2 a = Xa[N - pos], b = Xb[N - pos];   // conj(a) + i conj(b)
        return make_float2(a.x + b.y, b.x - a.y);
    }
    return make_float2(0.f, 0.f);
}

// Forward transform of two real rows held as v (first-pass order), then the
// half spectra of both rows for kz < NZ written to dstA, dstB (dstB may be
// null: single real row in v.x).
template <int N>
__device__ __forceinline__ void forward_pair_store(float2 *v, int p, int r, const float2 *tw, float2 *buf,
                                                   float2 *dstA, float2 *dstB, int NZ, bool row_ok)
{
    using PI = WPlanInfo<N>;
    constexpr int V = PI::V, P = PI::P;
    auto at = [&](int pos) { return row_slot<N>(buf, r, pos); };
    fft_line_warp<N, true>(v, p, tw, at);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < V; ++i) *at(PI::out_pos(p, i)) = v[i];
    __syncwarp();
    if (row_ok) {
        for (int k = p; k < NZ; k += P) {
            const float2 z = *at(k);
            const float2 w = cconj(*at(k == 0 ? 0 : N - k));
            // Xa = (Z_k + conj Z_{N-k}) / 2 ; Xb = (Z_k - conj Z_{N-k}) / (2i)
            dstA[k] = make_float2(0.5f * (z.x + w.x), 0.5f * (z.y + w.y));
            if (dstB) dstB[k] = make_float2(0.5f * (z.y - w.y), -0.5f * (z.x - w.x));
        }
    }
}

// MODE 0: nonlinear term (fields 0..5 of B -> fields 0..2 of B, in place)
// MODE 1: initial white noise (seeded, no input) -> fields 0..2 of B
// MODE 3: velocity to physical space: fields 0..2 of B -> A as reals [3][x][y][z]
// MODE 4: physical reals in A [3][x][y][z] -> forward along z into B fields 0..2
// grid (N*N/RZ, members), block RZ*P.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float white_noise(uint64_t seed, uint64_t counter)
{
    const double u1 = ((double)(splitmix64_at(seed, 2 * counter) >> 11) + 1.0) * 0x1.0p-53;
    const double u2 = ((double)(splitmix64_at(seed, 2 * counter + 1) >> 11) + 1.0) * 0x1.0p-53;
    return (float)(sqrt(-2.0 * log(u1)) * cospi(2.0 * u2));
}

template <int N, int MODE>
__global__ void __launch_bounds__(256, 2)
k_z(Geo g, MemberDev *md, int stage)
{
    using PI = WPlanInfo<N>;
    using RC = RowCfg<N>;
    constexpr int P = PI::P, V = PI::V, RZ = RC::RZ;
    extern __shared__ __align__(16) float2 sm[];
    float2 *tw = sm, *buf = sm + N;
    load_twiddles(tw, g.tw, N);
    const int p = threadIdx.x % P, r = threadIdx.x / P;
    const int m = blockIdx.y;
    const long long rho = (long long)blockIdx.x * RZ + r;   // row = y*N + x
    const int yy = (int)(rho / N), xx = (int)(rho % N);
    float2 *B = g.B + (long long)m * kFields * Dims<N>::SB + rho * Dims<N>::NZP;
    auto at = [&](int pos) { return row_slot<N>(buf, r, pos); };

    float2 w0[V], w1[V];   // forward inputs in first-pass order
    if constexpr (MODE == 0 || MODE == 3) {
        float2 a[V], b[V], cc[V];
        // all loads first (memory-level parallelism), then the transforms
#pragma unroll
        for (int i = 0; i < V; ++i) a[i] = pair_at(B, B + Dims<N>::SB, PI::in_pos(p, i), N, Dims<N>::KC);
        if constexpr (MODE == 3) {
#pragma unroll
            for (int i = 0; i < V; ++i) b[i] = pair_at(B + 2 * Dims<N>::SB, B + 2 * Dims<N>::SB, PI::in_pos(p, i), N, Dims<N>::KC);
        } else {
#pragma unroll
            for (int i = 0; i < V; ++i) b[i] = pair_at(B + 2 * Dims<N>::SB, B + 3 * Dims<N>::SB, PI::in_pos(p, i), N, Dims<N>::KC);
#pragma unroll
            for (int i = 0; i < V; ++i) cc[i] = pair_at(B + 4 * Dims<N>::SB, B + 5 * Dims<N>::SB, PI::in_pos(p, i), N, Dims<N>::KC);
        }
        fft_line_warp<N, false>(a, p, tw, at);
        fft_line_warp<N, false>(b, p, tw, at);
        if constexpr (MODE == 3) {
            // physical u_c(x, y, z) into A viewed as floats [member][3][x][y][z]
            float *out = reinterpret_cast<float *>(g.A + (long long)m * kFields * Dims<N>::SA);
            const long long n3 = (long long)N * N * N;
            const long long base = ((long long)xx * N + yy) * N;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const int q = PI::out_pos(p, i);
                out[base + q] = a[i].x;
                out[n3 + base + q] = a[i].y;
                out[2 * n3 + base + q] = b[i].x;
            }
            return;
        } else {
            fft_line_warp<N, false>(cc, p, tw, at);
            // a = ux + i uy, b = uz + i wx, cc = wy + i wz at positions out_pos
            float umax = 0.f;
            bool finite = true;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const float ux = a[i].x, uy = a[i].y, uz = b[i].x;
                const float wx = b[i].y, wy = cc[i].x, wz = cc[i].y;
                umax = fmaxf(umax, fmaxf(fabsf(ux), fmaxf(fabsf(uy), fabsf(uz))));
                finite = finite && isfinite(ux + uy + uz + wx + wy + wz);
                w0[i] = make_float2(uy * wz - uz * wy, uz * wx - ux * wz);
                w1[i] = make_float2(ux * wy - uy * wx, 0.f);
            }
            // block max of |u| -> member slot of this stage
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
            const unsigned ballot = __ballot_sync(0xffffffffu, !finite);
            if ((threadIdx.x & 31) == 0) {
                atomicMax(&md[g.first + m].umax_bits[stage], __float_as_uint(umax));
                if (ballot) atomicOr(&md[g.first + m].flags, kFlagNonFinite);
            }
            if constexpr (!PI::matched) {
                // reorder from last-pass positions to first-pass positions
                __syncwarp();
#pragma unroll
                for (int i = 0; i < V; ++i) *at(PI::out_pos(p, i)) = w0[i];
                __syncwarp();
#pragma unroll
                for (int i = 0; i < V; ++i) w0[i] = *at(PI::in_pos(p, i));
                __syncwarp();
#pragma unroll
                for (int i = 0; i < V; ++i) *at(PI::out_pos(p, i)) = w1[i];
                __syncwarp();
#pragma unroll
                for (int i = 0; i < V; ++i) w1[i] = *at(PI::in_pos(p, i));
            }
        }
    } else if constexpr (MODE == 1) {
        const uint64_t seed = (uint64_t)md[g.first + m].seed;
        const uint64_t n3 = (uint64_t)N * N * N;
        const uint64_t base = ((uint64_t)xx * N + yy) * N;
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const uint64_t idx = base + PI::in_pos(p, i);
            w0[i] = make_float2(white_noise(seed, idx), white_noise(seed, n3 + idx));
            w1[i] = make_float2(white_noise(seed, 2 * n3 + idx), 0.f);
        }
    } else if constexpr (MODE == 4) {
        const float *in = reinterpret_cast<const float *>(g.A + (long long)m * kFields * Dims<N>::SA);
        const long long n3 = (long long)N * N * N;
        const long long base = ((long long)xx * N + yy) * N;
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const int q = PI::in_pos(p, i);
            w0[i] = make_float2(in[base + q], in[n3 + base + q]);
            w1[i] = make_float2(in[2 * n3 + base + q], 0.f);
        }
    }
    if constexpr (MODE == 1 || MODE == 4) {
        __syncwarp();   // all threads reach the stores below after their loads
    }
    forward_pair_store<N>(w0, p, r, tw, buf, B, B + Dims<N>::SB, Dims<N>::NZ, true);
    forward_pair_store<N>(w1, p, r, tw, buf, B + 2 * Dims<N>::SB, nullptr, Dims<N>::NZ, true);
}

// ---------------------------------------------------------------------------
// FXU: forward along x of B-derived A fields 0..2, then per kept mode:
//   MODE 0: RK stage update (IF-SSP-RK2/3) of the state, FP64 partial sums
//   MODE 1: write F = P N + f into S (right-hand side, for checks)
//   MODE 2: initial field: write the projected noise spectrum to U and
//           accumulate shell energies
//   MODE 3: write the normalised forward transform (no projection) to U
// grid (NK*NZp/T, members), block T*P.
// ---------------------------------------------------------------------------
struct StageCoef {
    float a, ha, b, hb;   // out = a E(ha dt) u^n + b E(hb dt) (u^s + dt F)
};

__device__ __forceinline__ StageCoef stage_coef(int rk, int stage)
{
    if (rk == 2) {
        if (stage == 0) return {0.f, 0.f, 1.f, 1.f};
        return {0.5f, 1.f, 0.5f, 0.f};
    }
    if (stage == 0) return {0.f, 0.f, 1.f, 1.f};
    if (stage == 1) return {0.75f, 0.5f, 0.25f, -0.5f};
    // 1/3 and 2/3 are not binary fractions: with both rounded to FP32 their
    // sum is 1 + 3e-8, and the last stage would scale the state by that
    // factor every step (an energy drift of about 6e-8 per step).  a = 1 - b
    // is exact in FP32, so the weights sum to exactly 1.
    return {1.f - 2.f / 3.f, 1.f, 2.f / 3.f, 0.5f};
}

// Integrating factors of a stage, E(h dt) = exp(-nu k^2 h dt), kept as
// E - 1 (expm1) and applied as r + (E - 1) r.  Near k = 0 the factor is
// within a few FP32 ulps of 1: rounded to FP32 it would carry a relative
// error of up to ulp / (nu k^2 h dt) in the decay it applies -- for a capped
// dt the same error every step, a drift of the energy-containing modes.  In
// this form the decay increment keeps FP32 relative precision.
struct IfCoef {
    float a, ma, b, mb;   // out = a (u^n + ma u^n) + b (r + mb r)
};

__device__ __forceinline__ IfCoef if_coef(const StageCoef &co, float nu, float k2, float dt)
{
    return {co.a, co.a != 0.f ? expm1f(-nu * k2 * co.ha * dt) : 0.f, co.b, expm1f(-nu * k2 * co.hb * dt)};
}

__device__ __forceinline__ float if_combine(const IfCoef &c, float un, float r)
{
    return c.a * fmaf(c.ma, un, un) + c.b * fmaf(c.mb, r, r);
}

__device__ __forceinline__ double member_dt(const MemberDev &d, int N)
{
    if (d.dt_fixed > 0.0) return d.dt_fixed;
    const double umax = (double)__uint_as_float(d.umax_bits[0]);
    double dt = d.cfl * (2.0 * 3.14159265358979323846 / N) / umax;
    if (d.dt_max > 0.0 && dt > d.dt_max) dt = d.dt_max;
    return dt;
}

// End of an RK stage for member gm (one warp, lane = 0..31): the FP64
// partial sums of the update pass -> E, dissipation, band energy, the forcing
// amplitude alpha = eps_inj / (2 E_B) of the next stage, the CFL step after the
// first stage, time and step count after the last.
__device__ __forceinline__ void finish_body(MemberDev *md, const double *partial, int partial_blocks, int stage,
                                            int last_stage, int mode, int gm, int lane)
{
    MemberDev &d = md[gm];
    double e = 0.0, s = 0.0, b = 0.0;
    const double *pp = partial + (long long)gm * partial_blocks * 4;
    for (int k = lane; k < d.nblk; k += 32) {
        e += pp[k * 4 + 0];
        s += pp[k * 4 + 1];
        b += pp[k * 4 + 2];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        s += __shfl_xor_sync(0xffffffffu, s, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane != 0) return;
    if (mode == 0 && stage == 0) d.dt = member_dt(d, d.N);
    // injected power of the stage just taken: alpha(u^s) * 2 E_B(u^s)
    if (mode == 0) d.P = d.alpha * 2.0 * d.EB;
    d.E = e;
    d.diss = s;
    d.EB = b;
    // a non-finite value anywhere in the fields reaches every mode through
    // the nonlinear term and the transforms, hence these sums
    if (!isfinite(e) || !isfinite(s)) d.flags |= kFlagNonFinite;
    if (b > 0.0) {
        d.alpha = d.eps_inj / (2.0 * b);
    } else {
        d.alpha = 0.0;
        d.flags |= kFlagNoBandEnergy;
    }
    if (mode == 0 && last_stage) {
        d.t += d.dt;
        d.steps += 1;
        d.umax = (double)__uint_as_float(d.umax_bits[0]);
        for (int q = 0; q < 4; ++q) d.umax_bits[q] = 0u;
    }
}

template <int NW>
__device__ __forceinline__ void block_sum_to(double *out, double (&vals)[NW], double *scratch)
{
    // scratch: (blockDim/32) * NW doubles
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        double v = vals[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        vals[q] = v;
    }
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int q = 0; q < NW; ++q) scratch[warp * NW + q] = vals[q];
    }
    __syncthreads();
    if (threadIdx.x < NW) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += scratch[w * NW + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

template <int N, int MODE, int T, int VAR = 0>
__device__ __forceinline__ void fwd_x_body(const Geo &g, MemberDev *md, int stage, int last_stage, int bx, int m,
                                           float2 *sm)
{
    using PI = PlanInfo<N, VAR>;
    constexpr int P = PI::P, V = PI::V;
    float2 *tw = sm, *buf = sm + N, *tile = buf + N * T;   // tile: [3][NK][T]
    load_twiddles(tw, g.tw, N);
    const int c = threadIdx.x % T, p = threadIdx.x / T;
    const int col0 = bx * T;
    const int col = col0 + c;                                  // (ky, kz) flat
    const int iy = col / Dims<N>::NZP, kz = col % Dims<N>::NZP;
    const int kz0 = col0 % Dims<N>::NZP;                  // first kz of the tile
    const bool valid = kz < Dims<N>::NZ;
    constexpr int per = Dims<N>::NK * T;
    const float2 *Ain = g.A + (long long)m * kFields * Dims<N>::SA + ((long long)iy * N) * Dims<N>::NZP + kz;
    auto at = [&](int pos) { return &buf[pos * T + c]; };
    // forward transforms of the three components; kept rows to the tile.
    // The next component's inputs are loaded while this one is transformed.
    float2 v[V], nxt[V];
#pragma unroll
    for (int i = 0; i < V; ++i)
        v[i] = valid ? Ain[(long long)PI::in_pos(p, i) * Dims<N>::NZP] : make_float2(0.f, 0.f);
#pragma unroll 1
    for (int q = 0; q < 3; ++q) {
        if (q < 2) {
#pragma unroll
            for (int i = 0; i < V; ++i)
                nxt[i] = valid ? Ain[(long long)(q + 1) * Dims<N>::SA + (long long)PI::in_pos(p, i) * Dims<N>::NZP]
                               : make_float2(0.f, 0.f);
        }
        fft_line<N, true, VAR>(v, p, tw, at);
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const int kx = wnum(PI::out_pos(p, i), N);
            if (kx >= -Dims<N>::KC && kx <= Dims<N>::KC) tile[q * per + (kx >= 0 ? kx : kx + Dims<N>::NK) * T + c] = v[i];
        }
        if (q < 2) {
#pragma unroll
            for (int i = 0; i < V; ++i) v[i] = nxt[i];
        }
    }
    __syncthreads();

    const MemberDev &d = md[g.first + m];
    const float inv_n3 = 1.0f / ((float)N * (float)N * (float)N);
    const long long rowU = (long long)Dims<N>::NK * Dims<N>::NZP;
    float2 *U = g.U + (long long)m * 3 * Dims<N>::SU + col0;
    float2 *S = g.S + (long long)m * 3 * Dims<N>::SU + col0;
    const int kyi = iy <= Dims<N>::KC ? iy : iy - Dims<N>::NK;
    float se = 0.f, sd = 0.f, sb = 0.f;
    float dtf = 0.f, alpha = 0.f, nu = 0.f;
    StageCoef co{};
    if constexpr (MODE == 0 || MODE == 1) {
        dtf = (float)member_dt(d, N);
        alpha = (float)d.alpha;
        nu = (float)d.nu;
        co = stage_coef(d.rk, stage);
    }
    const int blo = d.band_lo2, bhi = d.band_hi2;
    double *shell_smem = reinterpret_cast<double *>(buf);   // exchange buffer is free now (MODE 2)
    if constexpr (MODE == 2) {
        for (int s = threadIdx.x; s < g.shells; s += blockDim.x) shell_smem[s] = 0.0;
        __syncthreads();
    }
    // per kept mode of the tile: thread <-> (kx row, column), coalesced in the
    // column; the state reads of UB modes are issued together before use
    constexpr int UB = VAR == 0 ? 4 : 2;   // fewer batched state reads under the tighter register budget
    for (int base = threadIdx.x; base < per; base += UB * blockDim.x) {
        float2 unb[UB][3], usb[UB][3];
        if constexpr (MODE == 0 || MODE == 1) {
#pragma unroll
            for (int u = 0; u < UB; ++u) {
                const int idx = base + u * blockDim.x;
                const int cc = idx % T;
                const bool ok = idx < per && kz0 + cc < Dims<N>::NZ;
                const long long off = (long long)(idx / T) * rowU + cc;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    unb[u][q] = ok ? U[q * Dims<N>::SU + off] : make_float2(0.f, 0.f);
                    usb[u][q] = (ok && stage != 0) ? S[q * Dims<N>::SU + off] : unb[u][q];
                }
            }
        }
#pragma unroll
    for (int u = 0; u < UB; ++u) {
        const int idx = base + u * blockDim.x;
        if (idx >= per) continue;
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
        for (int q = 0; q < 3; ++q) n[q] = cscale(tile[q * per + idx], inv_n3);
        if (MODE != 3) {
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
        }
        const float wgt = kzc == 0 ? 1.f : 2.f;   // Hermitian multiplicity in the full spectrum
        if constexpr (MODE == 2 || MODE == 3) {
#pragma unroll
            for (int q = 0; q < 3; ++q) U[q * Dims<N>::SU + off] = n[q];
            if constexpr (MODE == 2) {
                const int s = (int)lrintf(sqrtf(k2));
                float a2 = 0.f;
#pragma unroll
                for (int q = 0; q < 3; ++q) a2 += n[q].x * n[q].x + n[q].y * n[q].y;
                atomicAdd(&shell_smem[s], 0.5 * (double)(wgt * a2));
            }
        } else {
            const bool band = k2i >= blo && k2i <= bhi;
            float2 us[3], un[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                un[q] = unb[u][q];
                us[q] = usb[u][q];
                if (band) n[q] = make_float2(n[q].x + alpha * us[q].x, n[q].y + alpha * us[q].y);
            }
            if constexpr (MODE == 1) {
#pragma unroll
                for (int q = 0; q < 3; ++q) S[q * Dims<N>::SU + off] = n[q];
            } else {
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
    }
    }
    if constexpr (MODE == 2) {
        __syncthreads();
        double *shell = g.shell + (long long)m * g.shells;
        for (int s = threadIdx.x; s < g.shells; s += blockDim.x)
            if (shell_smem[s] != 0.0) atomicAdd(&shell[s], shell_smem[s]);
    }
    if constexpr (MODE == 0) {
        __syncthreads();   // buf is reused as reduction scratch
        double vals[3] = {(double)se, (double)sd, (double)sb};
        double *out = g.partial + ((long long)(g.first + m) * g.partial_blocks + bx) * 4;
        block_sum_to<3>(out, vals, reinterpret_cast<double *>(buf));
    }
}

template <int N, int MODE, int T, int VAR = 0>
__global__ void __launch_bounds__(ColCfg<N, T, VAR>::threads, ColCfg<N, T, VAR>::min_blocks)
k_fwd_x(Geo g, MemberDev *md, int stage, int last_stage)
{
    extern __shared__ __align__(16) float2 sm[];
    fwd_x_body<N, MODE, T, VAR>(g, md, stage, last_stage, blockIdx.x, blockIdx.y, sm);
}

}  // namespace ens
