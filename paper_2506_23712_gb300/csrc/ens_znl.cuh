// ZNL: the z-direction pass of an RK stage, persistent and TMA-fed.
//
// Per (y, x) row of a member: the six half spectra (u, omega) along z are
// taken to physical space as three complex lines (two real rows per complex
// line, Hermitian extension), the rotational nonlinear term n = u x omega is
// formed point by point together with max|u_i| (CFL step, Sec. IV), and n
// goes straight back along z; the dealiased half spectra of n overwrite
// fields 0..2 of the row in buffer B (n_z of two consecutive rows of a
// warp's stream share one forward complex line).  Non-finite values are
// caught downstream, in the stage's energy sums (k_finish).
//
// Each warp owns a stream of row groups (32/P rows per group, P threads per
// row) and double-buffers their inputs in shared memory: one lane issues
// six 1D bulk copies (cp.async.bulk, TMA) per row into the idle buffer,
// completion counted on that buffer's mbarrier, while the whole warp
// transforms the other buffer.  Waits are bounded; a wait that gives up
// flags the member (ENS_ETIMEOUT) and the warp stops.
#pragma once

#include "ens_kernels.cuh"
#include "ens_tma.cuh"

namespace ens {

// Classes of the first-pass input slots of a Hermitian pair line (slot I
// holds positions c + p, p < P, c the position of lane 0): the first slot
// (c = 0, the kz = 0 mode sits in lane 0), all positions in the zero band
// KC < k < N - KC, positions in [1, N - KC) read forwards from the staged
// half spectrum, positions in (KC, N) read backwards (the mirror), or a
// slot that needs both (checked per lane).  The staged rows are zero past
// the copied modes, so the forward and backward reads need no checks.
enum : int { kSlotFirst, kSlotZero, kSlotFwd, kSlotBwd, kSlotMixed };

template <int N, int VAR>
__host__ __device__ constexpr int slot_class(int i)
{
    using PI = WPlanInfo<N, VAR>;
    const int P = PI::P, KC = kc_of_n(N);
    const int c = (i / PI::R0) * P + (i % PI::R0) * (N / PI::R0);
    if (c == 0) return P - 1 < N - KC ? kSlotFirst : kSlotMixed;
    if (c > KC && c + P - 1 < N - KC) return kSlotZero;
    if (c + P - 1 < N - KC) return kSlotFwd;
    if (c > KC) return kSlotBwd;
    return kSlotMixed;
}

// staged row pitch (float2, even): the copied modes, then zeros up to the
// furthest padded read of a forward or backward slot
template <int N, int VAR>
__host__ __device__ constexpr int stage_pitch()
{
    using PI = WPlanInfo<N, VAR>;
    const int P = PI::P, NZ = kc_of_n(N) + 1;
    int need = (NZ + 1) / 2 * 2;
    for (int i = 0; i < PI::V; ++i) {
        const int c = (i / PI::R0) * P + (i % PI::R0) * (N / PI::R0);
        const int k = slot_class<N, VAR>(i);
        if ((k == kSlotFirst || k == kSlotFwd) && c + P > need) need = c + P;
        if (k == kSlotBwd && N - c + 1 > need) need = N - c + 1;
    }
    return (need + 1) / 2 * 2;
}

template <int N, int VAR = 0>
struct ZCfg {
    using PI = WPlanInfo<N, VAR>;
    static constexpr int P = PI::P, V = PI::V, LPW = 32 / P;
    static constexpr int WPB = 8;                          // warps per CTA
    static constexpr int NZ = kc_of_n(N) + 1;
    static constexpr int NZ2 = (NZ + 1) / 2 * 2;           // copied row length (16-byte multiple)
    static constexpr int PITCH = stage_pitch<N, VAR>();     // staged row pitch, zero past NZ2
    static constexpr int STAGE = LPW * 6 * PITCH;          // float2 per warp buffer
    // the power-of-two plans use the per-exchange padded layouts, the
    // others the rows of RowCfg (XOR-swizzled)
    static constexpr bool PAD = WPadV<N, VAR>::on;
    static constexpr int SROW = PAD ? WPadV<N, VAR>::SROW : VAR == 0 ? RowCfg<N>::SROW : N + N / 16 + N / 32 + 1;
    static __device__ __forceinline__ float2 *slot(float2 *buf, int r, int pos)
    {
        if constexpr (VAR == 0) return row_slot<N>(buf, r, pos);
        else return &buf[r * SROW + pos + (pos >> 4)];
    }
    static constexpr size_t smem_bytes()
    {
        return sizeof(float2) * (size_t)N + sizeof(uint64_t) * 2 * WPB + sizeof(float2) * (size_t)WPB * 2 * STAGE +
               sizeof(float2) * (size_t)WPB * LPW * SROW;
    }
};

// forward transform of two real rows with register twiddles, then the half
// spectra of both rows (kz < NZ) to dstA / dstB (dstB null: one real row)
template <int N, int VAR>
__device__ __forceinline__ void forward_pair_store_tw(float2 *v, int p, int r, const WarpTw<N, VAR> &T, float2 *buf,
                                                      float2 *dstA, float2 *dstB, int NZ)
{
    using PI = WPlanInfo<N, VAR>;
    constexpr int V = PI::V, P = PI::P;
    auto at = [&](int pos) { return ZCfg<N, VAR>::slot(buf, r, pos); };
    fft_line_warp_tw<N, true, VAR>(v, p, T, at);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < V; ++i) *at(PI::out_pos(p, i)) = v[i];
    __syncwarp();
    for (int k = p; k < NZ; k += P) {
        const float2 z = *at(k);
        const float2 w = cconj(*at(k == 0 ? 0 : N - k));
        // Xa = (Z_k + conj Z_{N-k}) / 2 ; Xb = (Z_k - conj Z_{N-k}) / (2i)
        dstA[k] = make_float2(0.5f * (z.x + w.x), 0.5f * (z.y + w.y));
        if (dstB) dstB[k] = make_float2(0.5f * (z.y - w.y), -0.5f * (z.x - w.x));
    }
}

// First (inverse) pass inputs of a Hermitian pair line a + i b from the
// staged half spectra Xa, Xb (zero past the copied modes), by slot class.
// With an odd mode count the copy carries one element past the kept modes
// (index NZ, outside the spectrum): the one lane that reads it takes zero.
template <int N, int VAR, int I>
struct PairSlots {
    static __device__ __forceinline__ void load(float2 *v, const float2 *Xa, const float2 *Xb, int p)
    {
        using PI = WPlanInfo<N, VAR>;
        constexpr int P = PI::P, KC = Dims<N>::KC, NZ = KC + 1;
        constexpr bool odd = (NZ & 1) != 0;
        if constexpr (I < PI::V) {
            constexpr int c = (I / PI::R0) * P + (I % PI::R0) * (N / PI::R0);
            constexpr int k = slot_class<N, VAR>(I);
            if constexpr (k == kSlotZero) {
                v[I] = make_float2(0.f, 0.f);
            } else if constexpr (k == kSlotFirst || k == kSlotFwd) {
                float2 a = Xa[c + p], b = Xb[c + p];
                if constexpr (odd && c <= NZ && NZ < c + P) {
                    if (p == NZ - c) a = b = make_float2(0.f, 0.f);
                }
                if constexpr (k == kSlotFirst)   // kz = 0: real parts only (C2R convention)
                    v[I] = p == 0 ? make_float2(a.x, b.x) : make_float2(a.x - b.y, a.y + b.x);
                else
                    v[I] = make_float2(a.x - b.y, a.y + b.x);
            } else if constexpr (k == kSlotBwd) {
                float2 a = Xa[N - c - p], b = Xb[N - c - p];   // conj(a) + i conj(b)
                if constexpr (odd && N - c - P < NZ && NZ <= N - c) {
                    if (p == N - c - NZ) a = b = make_float2(0.f, 0.f);
                }
                v[I] = make_float2(a.x + b.y, b.x - a.y);
            } else {
                v[I] = pair_at(Xa, Xb, c + p, N, KC);
            }
            PairSlots<N, VAR, I + 1>::load(v, Xa, Xb, p);
        }
    }
};

// Forward transform of two real rows (padded layouts), then the half
// spectra of both rows (kz < NZ) to dstA / dstB (dstB null: one real row).
// The last pass leaves position p + P i in slot i of lane p, so Z_{N-k}
// for this lane's k = p + P i sits in lane (P - p) mod P (slot V - 1 - i,
// or V - i for lane 0) and comes over by shuffle.
template <int N, int VAR>
__device__ __forceinline__ void forward_pair_store_shfl(float2 *v, int p, int line, const WarpTw<N, VAR> &T,
                                                        float2 *row, float2 *dstA, float2 *dstB)
{
    using PI = WPlanInfo<N, VAR>;
    constexpr int P = PI::P, V = PI::V, NZ = Dims<N>::NZ;
    static_assert(PI::RL == V, "the last pass must hold one butterfly per lane");
    static_assert((NZ + P - 1) / P <= V, "unpacking rounds exceed the slots");
    fft_line_warp_pad<N, true, VAR>(v, p, T, row);
    const int src = line * P + ((P - p) & (P - 1));
#pragma unroll
    for (int i = 0; i < (NZ + P - 1) / P; ++i) {
        const float2 send = p == 0 ? v[(V - i) % V] : v[V - 1 - i];
        const float2 z = v[i];
        const float2 w = make_float2(__shfl_sync(0xffffffffu, send.x, src), -__shfl_sync(0xffffffffu, send.y, src));
        const int k = p + i * P;
        if (k < NZ) {
            // Xa = (Z_k + conj Z_{N-k}) / 2 ; Xb = (Z_k - conj Z_{N-k}) / (2i)
            dstA[k] = cscale_x2(0.5f, cadd_x2(z, w));
            if (dstB) {
                const float2 d = csub_x2(z, w);
                dstB[k] = make_float2(0.5f * d.y, -0.5f * d.x);
            }
        }
    }
}

// Body of the z pass over the row groups [first + warp, T) of the group's
// members (all members' row groups concatenated), stepping W per warp
// iteration: the persistent kernel passes first = blockIdx.x WPB and
// W = gridDim.x WPB over every row group; the persistent stage kernel
// (ens_persist.cu) passes one member's chunk of row groups with W = WPB and
// TASK set: the shared memory then serves other work next, so the warps
// invalidate their barriers at the end.
template <int N, int VAR = 0, bool TASK = false>
__device__ __forceinline__ void znl_body(const Geo &g, MemberDev *md, int stage_idx, long long first, long long W,
                                         long long T, unsigned char *smraw)
{
    using C = ZCfg<N, VAR>;
    using PI = WPlanInfo<N, VAR>;
    constexpr int P = C::P, V = C::V, LPW = C::LPW, NZ2 = C::NZ2;
    float2 *tw = reinterpret_cast<float2 *>(smraw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(tw + N);
    float2 *stage = reinterpret_cast<float2 *>(bars + 2 * C::WPB);
    float2 *rows = stage + C::WPB * 2 * C::STAGE;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int line = lane / P, p = lane % P;
    uint64_t *bar = bars + 2 * warp;
    float2 *st = stage + warp * 2 * C::STAGE;
    float2 *rowbuf = rows + warp * LPW * C::SROW;
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    load_twiddles(tw, g.tw, N);   // block barrier also publishes the barrier init
    WarpTw<N, VAR> TW;            // this lane's inter-pass twiddles, for every row it transforms
    TW.init(p, tw);

    const long long G = (long long)N * N / LPW;   // row groups per member
    long long grp = first + warp;
    const uint32_t bytes = (uint32_t)(LPW * 6 * NZ2 * sizeof(float2));
    const long long skip_gi = g.z_skip_member >= 0 ? g.z_skip_member * G : -1;   // failure test only
    auto skipped = [&](long long gi) { return gi == skip_gi; };
    auto issue = [&](long long gi, int b) {   // lane 0 only
        const long long m = gi / G, lg = gi % G;
        if (skipped(gi)) return;   // failure test: nothing in flight for this barrier
        const float2 *src = g.B + m * kFields * Dims<N>::SB + (lg * LPW) * Dims<N>::NZP;
        float2 *dst = st + b * C::STAGE;
        mbar_arrive_expect_tx(&bar[b], bytes);
#pragma unroll 1
        for (int l = 0; l < LPW; ++l)
#pragma unroll
            for (int f = 0; f < 6; ++f)
                bulk_g2s(dst + (l * 6 + f) * C::PITCH, src + f * Dims<N>::SB + l * Dims<N>::NZP,
                         NZ2 * (uint32_t)sizeof(float2), &bar[b]);
    };
    // zero tails of the staged rows (never written by the copies)
    constexpr int TAIL = C::PITCH - NZ2;
    if constexpr (TAIL > 0) {
        for (int e = lane; e < 2 * LPW * 6 * TAIL; e += 32) st[(e / TAIL) * C::PITCH + NZ2 + e % TAIL] = make_float2(0.f, 0.f);
        __syncwarp();
    }
    if (lane == 0 && grp < T) issue(grp, 0);

    auto at = [&](int pos) { return C::slot(rowbuf, line, pos); };
    float2 *myrow = rowbuf + line * C::SROW;   // this lane's line (padded layouts)
    auto fwd_pair = [&](float2 *v, float2 *dA, float2 *dB) {
        if constexpr (C::PAD) forward_pair_store_shfl<N, VAR>(v, p, line, TW, myrow, dA, dB);
        else forward_pair_store_tw<N, VAR>(v, p, line, TW, rowbuf, dA, dB, Dims<N>::NZ);
    };
    float umax = 0.f;
    long long cur_m = grp < T ? grp / G : 0;
    auto flush = [&](long long m) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
        if (lane == 0) atomicMax(&md[g.first + m].umax_bits[stage_idx], __float_as_uint(umax));
        umax = 0.f;
    };
    bool timed_out = false;
    int it = 0;
    // n_z of consecutive rows of this warp's stream are paired into one
    // complex line for the forward transform (three forward lines per two
    // rows instead of four): the first row's n_z waits in registers
    float nzp[V];
    float2 *pend = nullptr;   // field-2 destination of the waiting row (warp-uniform null / non-null)
    for (; grp < T; ++it, grp += W) {
        const int b = it & 1;
        const long long nxt = grp + W;
        if (lane == 0 && nxt < T) {
            fence_proxy_async_smem();   // this buffer's earlier reads precede the refill
            issue(nxt, b ^ 1);
        }
        if (!mbar_wait_warp(&bar[b], (uint32_t)((it >> 1) & 1), skipped(grp) ? g.z_skip_wait : kWaitIters)) {
            timed_out = true;
            break;
        }
        const long long m = grp / G, lg = grp % G;
        if (m != cur_m) {
            flush(cur_m);
            cur_m = m;
        }
        const long long rho = lg * LPW + line;
        const float2 *X = st + b * C::STAGE + line * 6 * C::PITCH;
        float2 a[V], bb[V], cc[V], w0[V];
        float nz[V];
        constexpr int R = C::PITCH;
        PairSlots<N, VAR, 0>::load(a, X, X + R, p);
        PairSlots<N, VAR, 0>::load(bb, X + 2 * R, X + 3 * R, p);
        PairSlots<N, VAR, 0>::load(cc, X + 4 * R, X + 5 * R, p);
        if constexpr (C::PAD) {
            fft_line_warp_pad<N, false, VAR>(a, p, TW, myrow);
            fft_line_warp_pad<N, false, VAR>(bb, p, TW, myrow);
            fft_line_warp_pad<N, false, VAR>(cc, p, TW, myrow);
        } else {
            fft_line_warp_tw<N, false, VAR>(a, p, TW, at);
            fft_line_warp_tw<N, false, VAR>(bb, p, TW, at);
            fft_line_warp_tw<N, false, VAR>(cc, p, TW, at);
        }
        // a = ux + i uy, bb = uz + i wx, cc = wy + i wz at positions out_pos;
        // the CFL step takes max|u_i| of the first stage only
        if (stage_idx == 0) {
#pragma unroll
            for (int i = 0; i < V; ++i) umax = fmaxf(umax, fmaxf(fabsf(a[i].x), fmaxf(fabsf(a[i].y), fabsf(bb[i].x))));
        }
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const float ux = a[i].x, uy = a[i].y, uz = bb[i].x;
            const float wx = bb[i].y, wy = cc[i].x, wz = cc[i].y;
            w0[i] = make_float2(uy * wz - uz * wy, uz * wx - ux * wz);
            nz[i] = ux * wy - uy * wx;
        }
        static_assert(PI::matched, "first and last radix must agree");
        float2 *Bout = g.B + m * kFields * Dims<N>::SB + rho * Dims<N>::NZP;
        fwd_pair(w0, Bout, Bout + Dims<N>::SB);
        if (pend) {
#pragma unroll
            for (int i = 0; i < V; ++i) w0[i] = make_float2(nzp[i], nz[i]);
            fwd_pair(w0, pend, Bout + 2 * Dims<N>::SB);
            pend = nullptr;
        } else {
#pragma unroll
            for (int i = 0; i < V; ++i) nzp[i] = nz[i];
            pend = Bout + 2 * Dims<N>::SB;
        }
        __syncwarp();   // all lanes are done with buffer b before it is refilled
    }
    if (pend && !timed_out) {   // an odd row count: the last n_z goes alone
        float2 w[V];
#pragma unroll
        for (int i = 0; i < V; ++i) w[i] = make_float2(nzp[i], 0.f);
        fwd_pair(w, pend, nullptr);
    }
    if (grp > first + warp || timed_out) flush(cur_m);
    if (timed_out) {
        // this warp's remaining row groups (this member's and those of every
        // later member of the group) stay unprocessed: flag them all
        if (lane == 0)
            for (long long m = grp / G; m <= (T - 1) / G; ++m) atomicOr(&md[g.first + m].flags, kFlagTimeout);
        // the refill of the other buffer may still be in flight: wait for it (bounded)
        if (grp + W < T) mbar_wait_warp(&bar[(it & 1) ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
    }
    if constexpr (TASK) {
        __syncwarp();
        if (lane == 0) {
            mbar_inval(&bar[0]);
            mbar_inval(&bar[1]);
        }
    }
}

template <int N, int VAR = 0>
__global__ void __launch_bounds__(256, VAR == 0 && ZCfg<N, VAR>::smem_bytes() <= 110 * 1024 ? 2 : 1)
k_znl(Geo g, MemberDev *md, int stage_idx)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr long long G = (long long)N * N / ZCfg<N, VAR>::LPW;   // row groups per member
    znl_body<N, VAR>(g, md, stage_idx, (long long)blockIdx.x * ZCfg<N, VAR>::WPB,
                     (long long)gridDim.x * ZCfg<N, VAR>::WPB, G * g.members, smraw);
}

}  // namespace ens
