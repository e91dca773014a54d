// Learned lambda-interpolant of the member statistics: a 4-layer MLP
// (width 256, SiLU) that models the per-lambda densities p(Q, R | lambda),
// p(log eps | lambda) and p(log omega^2 | lambda) as a softmax over the
// histogram bins, trained on the members' own histograms in BF16 with FP32
// accumulation, so that the lambda mixture (Sec. II, Eq. ensemble_hypothesis;
// Sec. IV, Eq. gaussian_lambda_pdf) can be evaluated on a fine lambda
// quadrature between the simulated lambda values.  The paper has no such
// component; the member-quadrature mixture (ens_mixture) stays the reference
// against which the surrogate's error is measured (Hellinger distance).
//
// All contractions run on the 5th-generation tensor cores (tcgen05.mma,
// kind::f16, BF16 operands from shared memory, FP32 accumulator in tensor
// memory).  One GEMM kernel serves every layer:
//   forward  Z_l  = H_{l-1} W_l^T          A = H [rows][in],  B = W  [out][in]
//   backward dH   = dZ_l W_l               A = dZ [rows][out], B = W^T [in][out]
//   gradient dW_l = dZ_l^T H_{l-1}         A = dZ^T [out][rows], B = H^T [in][rows] (split over rows)
#include "../../include/ens.h"
#include "ens_internal.h"
#include "ens_tc.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

namespace ens {

constexpr int kHid = 256;     // hidden width
constexpr int kIn = 64;       // input features (padded)
constexpr int kFeat = 31;     // used input features

// ---------------------------------------------------------------------------
// GEMM: C[M][N] (FP32) = A[M][K] * B[N][K]^T, BF16 K-major operands.
// CTA tile 128 x BN, K in blocks of 64; blockIdx.z splits K (partials at
// C + z * c_split).  M % 128 == 0, N % BN == 0, K per split % 64 == 0.
// ---------------------------------------------------------------------------
template <int BN>
__global__ void __launch_bounds__(128, 1)
k_gemm_tc(const __nv_bfloat16 *__restrict__ A, int lda, const __nv_bfloat16 *__restrict__ B, int ldb,
          float *__restrict__ C, int ldc, long long c_split, int k_per_split, int *err)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = sm;                  // 128 x 64 BF16
    unsigned char *sB = sm + 128 * 128;      // BN x 64 BF16
    uint64_t *bar = reinterpret_cast<uint64_t *>(sB + BN * 128);
    uint32_t *holder = reinterpret_cast<uint32_t *>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long m0 = (long long)blockIdx.x * 128, n0 = (long long)blockIdx.y * BN;
    const long long k0 = (long long)blockIdx.z * k_per_split;
    if (warp == 0) tmem_alloc(holder, BN);
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *holder;
    constexpr uint32_t idesc = idesc_bf16(128, BN);
    bool ok = true;
    const int nkb = k_per_split / 64;
    int kb = 0;
    for (; kb < nkb; ++kb) {
        for (int idx = tid; idx < 128 * 8; idx += 128) {
            const int r = idx >> 3, ch = idx & 7;
            const uint4 v = *reinterpret_cast<const uint4 *>(A + (m0 + r) * lda + k0 + kb * 64 + ch * 8);
            *reinterpret_cast<uint4 *>(sA + r * 128 + ((ch ^ (r & 7)) << 4)) = v;
        }
        for (int idx = tid; idx < BN * 8; idx += 128) {
            const int r = idx >> 3, ch = idx & 7;
            const uint4 v = *reinterpret_cast<const uint4 *>(B + (n0 + r) * ldb + k0 + kb * 64 + ch * 8);
            *reinterpret_cast<uint4 *>(sB + r * 128 + ((ch ^ (r & 7)) << 4)) = v;
        }
        fence_proxy_async_smem();   // generic shared stores -> tensor-core (async proxy) reads
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint64_t da = desc_sw128(sA), db = desc_sw128(sB);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                tc_mma_bf16(taddr, da + 2 * k, db + 2 * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
            tc_commit(bar);
        }
        ok = mbar_wait_warp(bar, (uint32_t)(kb & 1));
        tc_fence_after();
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
    }
    if (ok) {
        const long long row = m0 + warp * 32 + lane;
        float *crow = C + blockIdx.z * c_split + row * ldc + n0;
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
            float v[32];
            tc_ld_32cols(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int i = 0; i < 32; i += 4)
                *reinterpret_cast<float4 *>(crow + c + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        }
    } else {
        if (tid == 0) atomicExch(err, 1);
        // the MMAs of the stuck k-block may still be running: wait (bounded) before freeing
        mbar_wait_warp(bar, (uint32_t)(kb & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, BN);
}

// dynamic shared memory: alignment slack, the two operand tiles, barrier and
// TMEM holder, plus 48 KB of unused headroom past the tiles
template <int BN>
constexpr size_t gemm_smem() { return 1024 + 128 * 128 + BN * 128 + 64 + 48 * 1024; }

static cudaError_t gemm_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<256>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gemm_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<128>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gemm_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<64>());
    return e;
}

// C = A B^T with optional split of K; returns false on an unsupported shape
static bool gemm(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, float *C, int ldc, int M, int N,
                 int K, int ksplit, int *err, cudaStream_t s)
{
    if (M % 128 || K % (64 * ksplit) || ksplit < 1) return false;
    const int kps = K / ksplit;
    const long long cs = (long long)M * ldc;
    if (N % 256 == 0) {
        dim3 grid(M / 128, N / 256, ksplit);
        k_gemm_tc<256><<<grid, 128, gemm_smem<256>(), s>>>(A, lda, B, ldb, C, ldc, cs, kps, err);
    } else if (N % 128 == 0) {
        dim3 grid(M / 128, N / 128, ksplit);
        k_gemm_tc<128><<<grid, 128, gemm_smem<128>(), s>>>(A, lda, B, ldb, C, ldc, cs, kps, err);
    } else if (N % 64 == 0) {
        dim3 grid(M / 128, N / 64, ksplit);
        k_gemm_tc<64><<<grid, 128, gemm_smem<64>(), s>>>(A, lda, B, ldb, C, ldc, cs, kps, err);
    } else {
        return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// MLP pieces (CUDA cores)
// ---------------------------------------------------------------------------
struct RowSpec {
    int nq, nt;          // bins of the Q-R histogram per axis and of each tail histogram
    int per_member;      // nq*nq + 2*nt rows per lambda value
};

// input features of (lambda, bin): scaled bin coordinates, lambda / 5, the
// PDF kind, and sin/cos(pi k s) of the bin coordinates for k = 1..4
__device__ void row_features(const RowSpec &rs, double lam, int bin, float *f)
{
    for (int i = 0; i < kIn; ++i) f[i] = 0.f;
    float q = 0.f, r = 0.f, x = 0.f;
    int kind;
    if (bin < rs.nq * rs.nq) {
        kind = 0;
        q = (float)(((bin / rs.nq) + 0.5) / rs.nq * 2.0 - 1.0);
        r = (float)(((bin % rs.nq) + 0.5) / rs.nq * 2.0 - 1.0);
    } else {
        const int b = bin - rs.nq * rs.nq;
        kind = b < rs.nt ? 1 : 2;
        x = (float)(((b % rs.nt) + 0.5) / rs.nt * 2.0 - 1.0);
    }
    f[0] = q;
    f[1] = r;
    f[2] = (float)(lam / 5.0);
    f[3] = x;
    f[4] = kind == 0 ? 1.f : 0.f;   // one-hot kind, compile-time slots (keeps f in registers)
    f[5] = kind == 1 ? 1.f : 0.f;
    f[6] = kind == 2 ? 1.f : 0.f;
    const float s3[3] = {q, r, x};
    int o = 7;
    for (int c = 0; c < 3; ++c) {
        // sin, cos (pi k s), k = 1..4: one evaluation, then the angle-addition
        // recurrence sin((k+1) a) = sin(k a) cos a + cos(k a) sin a (and the
        // cosine likewise); far below the BF16 rounding of the features
        float s1, c1;
        sincospif(s3[c], &s1, &c1);
        float sk = s1, ck = c1;
#pragma unroll
        for (int k = 1; k <= 4; ++k) {
            f[o++] = sk;
            f[o++] = ck;
            const float sn = fmaf(sk, c1, ck * s1), cn = fmaf(ck, c1, -sk * s1);
            sk = sn;
            ck = cn;
        }
    }
}

__global__ void k_features(RowSpec rs, const double *lams, int nlam, long long rows_pad, __nv_bfloat16 *X,
                           __nv_bfloat16 *Xt)
{
    const long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= rows_pad) return;
    float f[kIn];
    const long long real = (long long)nlam * rs.per_member;
    if (row < real) {
        row_features(rs, lams[row / rs.per_member], (int)(row % rs.per_member), f);
    } else {
        for (int i = 0; i < kIn; ++i) f[i] = 0.f;
    }
    for (int i = 0; i < kIn; ++i) {
        X[row * kIn + i] = __float2bfloat16(f[i]);
        if (Xt) Xt[(long long)i * rows_pad + row] = __float2bfloat16(f[i]);
    }
}

// sigmoid(z) = (1 + tanh(z/2)) / 2 with the hardware tanh approximation: one
// special-function-unit operation per element (the epilogues are bound by
// that unit), relative error far below the BF16 rounding of the activations
__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sigmoid(float z) { return fmaf(0.5f, tanh_approx(0.5f * z), 0.5f); }
// SiLU z sigmoid(z) written with h = z / 2 as h + h tanh(h): two FMAs and one
// tanh (the fused inference forms h = v / 2 + b / 2 in one FMA with halved
// biases, bit for bit the same h as (v + b) / 2)
__device__ __forceinline__ float silu_h(float h) { return fmaf(h, tanh_approx(h), h); }
__device__ __forceinline__ float silu(float z) { return silu_h(0.5f * z); }
__device__ __forceinline__ float dsilu(float z)
{
    const float s = sigmoid(z);
    return s * (1.f + z * (1.f - s));
}

// BF16 rounding (round to nearest, ties to even) on the integer pipe: the
// upper 16 bits of the result are the BF16 of f, bit for bit the conversion
// instruction's result for every non-NaN f (a NaN stays a NaN).
__device__ __forceinline__ uint32_t bf16_rne_bits(float f)
{
    const uint32_t u = __float_as_uint(f);
    return u + 0x7FFFu + ((u >> 16) & 1u);
}
// two BF16 values in one word: lo in bits 0..15, hi in bits 16..31
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    return __byte_perm(bf16_rne_bits(lo), bf16_rne_bits(hi), 0x7632);
}
// the same with the conversion instruction (round to nearest even, one
// instruction for the pair): the fused inference's epilogues, where it
// measured faster than the integer-pipe form
__device__ __forceinline__ uint32_t cvt_bf16x2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
// f rounded to BF16, as FP32
__device__ __forceinline__ float round_bf16(float f) { return __uint_as_float(bf16_rne_bits(f) & 0xFFFF0000u); }

// a * b + c on both halves with one packed FP32x2 instruction (each half
// rounded as the scalar FMA)
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(r)
        : "l"(*reinterpret_cast<const unsigned long long *>(&a)), "l"(*reinterpret_cast<const unsigned long long *>(&b)),
          "l"(*reinterpret_cast<const unsigned long long *>(&c)));
    return *reinterpret_cast<const float2 *>(&r);
}
// SiLU of two pre-activations in the halved form h = (z + b) / 2 (see
// silu_h): the FMAs packed, one hardware tanh per element
__device__ __forceinline__ float2 silu_pair(float2 v, float2 bh)
{
    const float2 h = fma2(make_float2(0.5f, 0.5f), v, bh);
    return fma2(h, make_float2(tanh_approx(h.x), tanh_approx(h.y)), h);
}

// Z += bias (kept, FP32, for the backward pass); H = SiLU(Z) as BF16 (and H^T)
__global__ void k_bias_silu(float *Z, const float *bias, long long rows, __nv_bfloat16 *H, __nv_bfloat16 *Ht)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * kHid) return;
    const long long row = i / kHid;
    const int c = (int)(i % kHid);
    const float z = Z[i] + bias[c];
    Z[i] = z;
    const __nv_bfloat16 h = __float2bfloat16(silu(z));
    H[i] = h;
    if (Ht) Ht[(long long)c * rows + row] = h;
}

// logit = H3 . w4 + b4, one warp per row
__global__ void k_head(const __nv_bfloat16 *H, const float *w4, const float *b4, long long rows, float *logit)
{
    const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    float s = 0.f;
    for (int c = lane; c < kHid; c += 32) s += __bfloat162float(H[row * kHid + c]) * w4[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) logit[row] = s + b4[0];
}

// Per group (one lambda value and one PDF kind): log-softmax over its bins,
// densities q, cross-entropy against the target probabilities p (optional),
// dlogit = (q - p) * weight.  One block per group.
__global__ void k_softmax_ce(const float *logit, const float *target, int nq, int nt, double weight, float *q,
                             float *dlogit, double *loss_partial)
{
    const int g = blockIdx.x;
    const int member = g / 3, kind = g % 3;
    const int per = nq * nq + 2 * nt;
    const long long off = (long long)member * per + (kind == 0 ? 0 : nq * nq + (kind - 1) * nt);
    const int len = kind == 0 ? nq * nq : nt;
    __shared__ float red[32];
    __shared__ float bval;
    float mx = -INFINITY;
    for (int i = threadIdx.x; i < len; i += blockDim.x) mx = fmaxf(mx, logit[off + i]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        bval = m;
    }
    __syncthreads();
    mx = bval;
    float se = 0.f;
    for (int i = threadIdx.x; i < len; i += blockDim.x) se += __expf(logit[off + i] - mx);
    for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = se;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        bval = s;
    }
    __syncthreads();
    const float lse = mx + __logf(bval);
    float l = 0.f;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const float lq = logit[off + i] - lse;
        const float qi = __expf(lq);
        if (q) q[off + i] = qi;
        if (target) {
            const float p = target[off + i];
            if (p > 0.f) l -= p * lq;
            if (dlogit) dlogit[off + i] = (float)((qi - p) * weight);
        }
    }
    if (loss_partial) {
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
            loss_partial[g] = s * weight;
        }
    }
}

// dZ3 = (dlogit w4^T) * SiLU'(Z3) as BF16 (and dZ3^T); rows beyond `real` are zero
__global__ void k_head_back(const float *dlogit, const float *w4, const float *Z, long long rows, long long real,
                            __nv_bfloat16 *dZ, __nv_bfloat16 *dZt)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * kHid) return;
    const long long row = i / kHid;
    const int c = (int)(i % kHid);
    const float v = row < real ? dlogit[row] * w4[c] * dsilu(Z[i]) : 0.f;
    const __nv_bfloat16 b = __float2bfloat16(v);
    dZ[i] = b;
    dZt[(long long)c * rows + row] = b;
}

// dZ = dH * SiLU'(Z) as BF16 (and dZ^T)
__global__ void k_silu_back(const float *dH, const float *Z, long long rows, __nv_bfloat16 *dZ, __nv_bfloat16 *dZt)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * kHid) return;
    const long long row = i / kHid;
    const int c = (int)(i % kHid);
    const __nv_bfloat16 b = __float2bfloat16(dH[i] * dsilu(Z[i]));
    dZ[i] = b;
    dZt[(long long)c * rows + row] = b;
}

// column sums over rows of a BF16 [rows][kHid] matrix (bias gradients) and
// of dlogit * H (head weight gradient), deterministic: one block per column
__global__ void k_colsum_bf16(const __nv_bfloat16 *M, long long rows, float *out)
{
    const int c = blockIdx.x;
    float s = 0.f;
    for (long long r = threadIdx.x; r < rows; r += blockDim.x) s += __bfloat162float(M[r * kHid + c]);
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        out[c] = t;
    }
}

__global__ void k_head_grad(const float *dlogit, const __nv_bfloat16 *H, long long real, float *gw4, float *gb4)
{
    const int c = blockIdx.x;   // 0..kHid (kHid: bias)
    float s = 0.f;
    for (long long r = threadIdx.x; r < real; r += blockDim.x)
        s += dlogit[r] * (c < kHid ? __bfloat162float(H[r * kHid + c]) : 1.f);
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        if (c < kHid) gw4[c] = t;
        else gb4[0] = t;
    }
}

// sum of split-K partials (fixed order)
__global__ void k_sum_splits(const float *part, int splits, long long n, float *out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[(long long)z * n + i];
    out[i] = s;
}

// Adam on the FP32 master parameters; refresh the BF16 operand copies
struct ParamLayout {
    long long W1, b1, W2, b2, W3, b3, w4, b4, total;
};

__host__ __device__ inline ParamLayout param_layout()
{
    ParamLayout L{};
    long long o = 0;
    L.W1 = o; o += (long long)kHid * kIn;
    L.b1 = o; o += kHid;
    L.W2 = o; o += (long long)kHid * kHid;
    L.b2 = o; o += kHid;
    L.W3 = o; o += (long long)kHid * kHid;
    L.b3 = o; o += kHid;
    L.w4 = o; o += kHid;
    L.b4 = o; o += 1;
    L.total = o;
    return L;
}

__global__ void k_adam(float *p, const float *g, float *m1, float *m2, long long n, float lr, float b1, float b2,
                       float eps, float bc1, float bc2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a / bc1) / (sqrtf(b / bc2) + eps);
}

// byte offset of W[o][k] in the shared-memory image of a [256 out][K in]
// weight: K-blocks of 64 (32 KB each: 256 rows x 128 bytes, 128-byte swizzle)
__device__ __forceinline__ uint32_t wimg_offset(int o, int k)
{
    return (uint32_t)((k >> 6) * 32768) + sw128_offset(o, k & 63);
}

// BF16 operand copies: W1 [256][64], W2/W3 [256][256] and their transposes,
// and (optional) the swizzled shared-memory images of W1, W2, W3 that the
// fused inference kernel copies in with bulk copies
__global__ void k_pack_weights_img(const float *p, unsigned char *img1, unsigned char *img2, unsigned char *img3)
{
    const ParamLayout L = param_layout();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (long long)kHid * kIn) {
        const int o = (int)(i / kIn), k = (int)(i % kIn);
        *reinterpret_cast<__nv_bfloat16 *>(img1 + wimg_offset(o, k)) = __float2bfloat16(p[L.W1 + i]);
    }
    if (i < (long long)kHid * kHid) {
        const int o = (int)(i / kHid), k = (int)(i % kHid);
        *reinterpret_cast<__nv_bfloat16 *>(img2 + wimg_offset(o, k)) = __float2bfloat16(p[L.W2 + i]);
        *reinterpret_cast<__nv_bfloat16 *>(img3 + wimg_offset(o, k)) = __float2bfloat16(p[L.W3 + i]);
    }
}

__global__ void k_pack_weights(const float *p, __nv_bfloat16 *W1b, __nv_bfloat16 *W2b, __nv_bfloat16 *W3b,
                               __nv_bfloat16 *W2t, __nv_bfloat16 *W3t)
{
    const ParamLayout L = param_layout();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (long long)kHid * kIn) W1b[i] = __float2bfloat16(p[L.W1 + i]);
    if (i < (long long)kHid * kHid) {
        const int o = (int)(i / kHid), c = (int)(i % kHid);
        const __nv_bfloat16 w2 = __float2bfloat16(p[L.W2 + i]), w3 = __float2bfloat16(p[L.W3 + i]);
        W2b[i] = w2;
        W3b[i] = w3;
        W2t[(long long)c * kHid + o] = w2;
        W3t[(long long)c * kHid + o] = w3;
    }
}

// mixture of the surrogate densities over a lambda quadrature:
// pdf(b) = sum_j w_j q(b | lambda_j) / width(b)
__global__ void k_quad_mix(const float *q, const double *w, int nlam, int per, int nq, double dq, double dr,
                           double dt, double *pdf)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= per) return;
    double s = 0.0;
    for (int j = 0; j < nlam; ++j) s += w[j] * (double)q[(long long)j * per + b];
    pdf[b] = s / (b < nq * nq ? dq * dr : dt);
}

__global__ void k_quad_weights(double lo, double hi, int n, int kind, double c, double Z, double mu, double sigma,
                               double *lam, double *w)
{
    // midpoint rule over [lo, hi]; cell masses of the lambda distribution
    __shared__ double tot;
    const double d = (hi - lo) / n;
    const double m = kind == 0 ? -4.5 * c * Z : mu;
    const double s = kind == 0 ? sqrt(9.0 * c * Z) : sigma;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double a = lo + j * d, b = a + d;
        lam[j] = a + 0.5 * d;
        const double za = (a - m) / s, zb = (b - m) / s;
        w[j] = za >= 0.0 ? 0.5 * (erfc(za * 0.70710678118654752440) - erfc(zb * 0.70710678118654752440))
                         : 0.5 * (erfc(-zb * 0.70710678118654752440) - erfc(-za * 0.70710678118654752440));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int j = 0; j < n; ++j) t += w[j];
        tot = t;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) w[j] = tot > 0.0 ? w[j] / tot : 0.0;
}

__global__ void k_init_params(float *p, long long n, unsigned long long seed)
{
    // He-style uniform init from a counter hash; biases zero
    const ParamLayout L = param_layout();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    const float u = (float)((z >> 40) * (1.0 / 16777216.0)) * 2.f - 1.f;
    float scale = 0.f;
    if (i >= L.W1 && i < L.b1) scale = sqrtf(6.f / kFeat);
    else if ((i >= L.W2 && i < L.b2) || (i >= L.W3 && i < L.b3)) scale = sqrtf(6.f / kHid);
    else if (i >= L.w4 && i < L.b4) scale = sqrtf(3.f / kHid);
    p[i] = u * scale;
}

// Feature rows of the fused inference: every bin's row with lambda = 0, as
// packed BF16 pairs (the row does not depend on lambda except for input 2),
// and per lambda value the BF16 of lambda / 5, which the kernel puts in
// place of input 2 (the low half of word 1): the same bits as computing the
// row for that lambda.
__global__ void k_feature_table(RowSpec rs, const double *lams, int nlam, uint4 *ftab, uint32_t *lam5)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nlam) lam5[i] = bf16_rne_bits((float)(lams[i] / 5.0)) >> 16;
    if (i >= rs.per_member) return;
    float f[kIn];
    row_features(rs, 0.0, i, f);
    uint32_t w[kIn / 2];
#pragma unroll
    for (int j = 0; j < kIn / 2; ++j) w[j] = pack_bf16x2(f[2 * j], f[2 * j + 1]);
#pragma unroll
    for (int j = 0; j < kIn / 8; ++j) ftab[(long long)i * (kIn / 8) + j] = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
}

// biases and head weights by value: kernel parameters live in the constant
// bank, read in pairs by the epilogues (warp-uniform addresses: broadcasts)
struct MlpBias {
    float b1[kHid], b2[kHid], b3[kHid];   // halved: the epilogues form (z + b) / 2 in one FMA
    float w4[kHid];
    float b4;
};

// ---------------------------------------------------------------------------
// Fused inference: features -> 3 x (tcgen05 GEMM + bias + SiLU) -> head, per
// 128-row tile; activations never leave the SM.  Persistent CTAs, two tiles
// in flight per CTA (tiles A and B of a tile pair), so that the tensor cores
// work on one tile while the epilogue warps work on the other.  Per CTA:
//   TMEM          one 256-column FP32 accumulator per tile (512 columns)
//   shared memory H_A, H_B: 4 K-blocks of 128 rows x 64 BF16 each (64 KB
//                 each; K-block 0 also holds the tile's features, K-block 1
//                 the head's partial sums); a ring of three 32 KB slots for
//                 the weight K-blocks, streamed in the order they are used
//                 (W1, W2 blocks 0-3, W3 blocks 0-3 per tile pair)
//   warps 0-15    epilogues, in the order E1(A) E1(B) E2(A) E2(B) head(A)
//                 head(B): TMEM -> bias + SiLU -> BF16 K-blocks of the next
//                 layer's A operand (one arrival per warp and chunk), the
//                 head's dot product with w4; the next pair's features
//   warp 16       MMA issue: per hidden layer A0 A1 A2 B0 B1 B2 A3 B3
//                 (K-block c of tile X once its chunk c is written and the
//                 block has landed); a weight slot is released by a commit
//                 after the B tile's MMAs on it
//   warp 17       bulk copies of the weight K-blocks into free slots
// An accumulator is reused by the next layer of its tile: every epilogue
// warp loads all four chunks of it before its first chunk arrival, so the
// next layer's first MMA (which overwrites it) waits on that arrival.
// Epilogue warp w reads TMEM lanes 32 (w mod 4) .. +31 (its rows) and, in
// chunk c, columns 64 c + 16 (w / 4) .. +15; SiLU(z + b) = h + h tanh(h)
// with h = z / 2 + b / 2 (halved biases), the activations rounded to BF16,
// the head's partial sums over each warp's columns added in a fixed order.
// Every wait is bounded; a role whose wait gives up leaves its loop, sets
// *err, and the CTA drains its copies and MMAs before freeing the TMEM.
// ---------------------------------------------------------------------------
constexpr int kPairWarps = 16;                           // epilogue warps
constexpr int kPairThreads = 32 * (kPairWarps + 2);      // + MMA warp + copy warp
constexpr int kPairSlots = 3;                            // weight K-block slots
constexpr size_t kPairSmem = 1024 + 2 * 65536 + (size_t)kPairSlots * 32768 + 256;

__global__ void __launch_bounds__(kPairThreads, 1)
k_mlp_infer_pair(RowSpec rs, const uint4 *__restrict__ ftab, const uint32_t *__restrict__ lam5, long long real,
                 long long ntiles, const unsigned char *__restrict__ img1, const unsigned char *__restrict__ img2,
                 const unsigned char *__restrict__ img3, const __grid_constant__ MlpBias bias,
                 float *__restrict__ logit, int *err)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *const sH0 = sm, *const sH1 = sm + 65536;   // H of tile A, B
    unsigned char *const sW = sm + 2 * 65536;                  // weight slots
    uint64_t *bars = reinterpret_cast<uint64_t *>(sW + kPairSlots * 32768);
    uint64_t *full = bars;                       // [3] slot holds its K-block
    uint64_t *empty = bars + 3;                  // [3] slot's MMAs done (both tiles)
    uint64_t *accr = bars + 6;                   // [2] a layer's MMAs of tile X done
    uint64_t *chunk = bars + 8;                  // [2][4] chunk c of tile X written
    uint64_t *feat = bars + 16;                  // [2] features written, accumulator read
    uint64_t *drain = bars + 18;                 // every issued MMA done
    uint64_t *partd = bars + 19;                 // [2] head partial sums of tile X written
    uint32_t *holder = reinterpret_cast<uint32_t *>(bars + 21);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tmem_alloc(holder, 512);
    if (tid == 0) {
        for (int s = 0; s < kPairSlots; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int x = 0; x < 2; ++x) {
            mbar_init(&accr[x], 1);
            mbar_init(&feat[x], kPairWarps);
            mbar_init(&partd[x], kPairWarps);
        }
        for (int i = 0; i < 8; ++i) mbar_init(&chunk[i], kPairWarps);
        mbar_init(drain, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *holder;
    const long long npairs = (ntiles + 1) / 2;
    auto slot = [&](long long q) { return sW + (int)(q % kPairSlots) * 32768; };
    bool ok = true;
    if (warp == kPairWarps + 1) {
        // ---- copy warp: K-block q of the sequence into slot q mod 3 once the
        // block that held it (q - 3) is released ----
        long long q = 0;
        long long lastq[kPairSlots] = {-1, -1, -1};
        for (long long p = blockIdx.x; ok && p < npairs; p += gridDim.x) {
            for (int j = 0; j < 9; ++j, ++q) {
                const int s = (int)(q % kPairSlots);
                if (q >= kPairSlots) ok = mbar_wait_warp(&empty[s], (uint32_t)(((q / kPairSlots) & 1) ^ 1));
                if (!ok) break;
                if (lane == 0) {
                    const unsigned char *src = j == 0 ? img1 : (j < 5 ? img2 + (j - 1) * 32768 : img3 + (j - 5) * 32768);
                    mbar_arrive_expect_tx(&full[s], 32768);
                    bulk_g2s(sW + s * 32768, src, 32768, &full[s]);
                }
                lastq[s] = q;
            }
        }
        if (!ok) {
            // the copies this warp issued complete before the CTA ends (bounded)
            for (int s = 0; s < kPairSlots; ++s)
                if (lastq[s] >= 0) mbar_wait_warp(&full[s], (uint32_t)((lastq[s] / kPairSlots) & 1));
        }
    } else if (warp == kPairWarps) {
        // ---- MMA warp ----
        constexpr uint32_t idesc = idesc_bf16(128, kHid);
        uint32_t nfeat[2] = {0, 0}, nchunk[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        long long q = 0;
        auto wfull = [&](long long qq) {
            return mbar_wait_warp(&full[qq % kPairSlots], (uint32_t)((qq / kPairSlots) & 1));
        };
        auto wchunk = [&](int x, int c) {
            const bool r = mbar_wait_warp(&chunk[4 * x + c], nchunk[4 * x + c] & 1);
            if (r) ++nchunk[4 * x + c];
            return r;
        };
        // the four K = 16 MMAs of one K-block of tile x (a: its A operand block)
        auto mma_kb = [&](int x, const unsigned char *a, const unsigned char *b, bool first) {
            if (lane == 0) {
                tc_fence_after();
                const uint64_t da = desc_sw128(a), db = desc_sw128(b);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    tc_mma_bf16(taddr + 256u * x, da + 2 * k, db + 2 * k, idesc, (!first || k > 0) ? 1u : 0u);
            }
            __syncwarp();
        };
        for (long long p = blockIdx.x; ok && p < npairs; p += gridDim.x) {
            // layer 1 (K = 64: one block, the features)
            ok = wfull(q) && mbar_wait_warp(&feat[0], nfeat[0] & 1);
            if (!ok) break;
            ++nfeat[0];
            mma_kb(0, sH0, slot(q), true);
            if (lane == 0) tc_commit(&accr[0]);
            ok = mbar_wait_warp(&feat[1], nfeat[1] & 1);
            if (!ok) break;
            ++nfeat[1];
            mma_kb(1, sH1, slot(q), true);
            if (lane == 0) {
                tc_commit(&accr[1]);
                tc_commit(&empty[q % kPairSlots]);
            }
            ++q;
            // layers 2 and 3: A0 A1 A2 B0 B1 B2 A3 B3
            for (int l = 0; l < 2 && ok; ++l, q += 4) {
                for (int c = 0; c < 3 && ok; ++c) {
                    ok = wfull(q + c) && wchunk(0, c);
                    if (ok) mma_kb(0, sH0 + c * 16384, slot(q + c), c == 0);
                }
                for (int c = 0; c < 3 && ok; ++c) {
                    ok = wchunk(1, c);
                    if (ok) {
                        mma_kb(1, sH1 + c * 16384, slot(q + c), c == 0);
                        if (lane == 0) tc_commit(&empty[(q + c) % kPairSlots]);
                    }
                }
                if (ok) ok = wfull(q + 3) && wchunk(0, 3);
                if (ok) {
                    mma_kb(0, sH0 + 3 * 16384, slot(q + 3), false);
                    if (lane == 0) tc_commit(&accr[0]);
                    ok = wchunk(1, 3);
                }
                if (ok) {
                    mma_kb(1, sH1 + 3 * 16384, slot(q + 3), false);
                    if (lane == 0) {
                        tc_commit(&accr[1]);
                        tc_commit(&empty[(q + 3) % kPairSlots]);
                    }
                }
            }
        }
        // every MMA this warp issued completes before the TMEM is freed (bounded)
        if (lane == 0) tc_commit(drain);
        __syncwarp();
        mbar_wait_warp(drain, 0);
    } else {
        // ---- epilogue warps ----
        const int quarter = warp & 3, cpart = warp >> 2;
        const int row = quarter * 32 + lane;                  // this thread's TMEM lane = tile row
        const uint32_t lanes = (uint32_t)(quarter * 32) << 16;
        uint32_t nacc[2] = {0, 0}, npart[2] = {0, 0};
        // the features of tile t into K-block 0 of H, spread over every
        // epilogue thread: row tid / 4, 16-byte words 2 (tid mod 4) and the
        // next one; the bin's row of the table with lambda / 5 in place of
        // input 2 (the low half of word 1)
        auto features = [&](long long t, unsigned char *H) {
            const int r = tid >> 2, j0 = (tid & 3) * 2;
            const long long rr = t * 128 + r;
            uint4 v0 = make_uint4(0u, 0u, 0u, 0u), v1 = v0;
            if (rr < real) {
                const int li = (int)(rr / rs.per_member);
                const long long bin = rr - (long long)li * rs.per_member;
                v0 = ftab[bin * (kIn / 8) + j0];
                v1 = ftab[bin * (kIn / 8) + j0 + 1];
                if (j0 == 0) v0.y = (v0.y & 0xFFFF0000u) | lam5[li];
            }
            *reinterpret_cast<uint4 *>(H + sw128_offset(r, 8 * j0)) = v0;
            *reinterpret_cast<uint4 *>(H + sw128_offset(r, 8 * j0 + 8)) = v1;
        };
        // the first pair's features
        features(2 * (long long)blockIdx.x, sH0);
        features(2 * (long long)blockIdx.x + 1, sH1);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(&feat[0]);
            mbar_arrive(&feat[1]);
        }
        // epilogue of a hidden layer of tile x (bias bv): H_x chunk c, arrival c
        // (every chunk's load is waited for before the first arrival: the
        // next layer's first MMA overwrites the whole accumulator)
        auto epilogue = [&](int x, const float *bv) {
            if (!(ok && mbar_wait_warp(&accr[x], nacc[x] & 1))) return false;
            ++nacc[x];
            tc_fence_after();
            unsigned char *H = x ? sH1 : sH0;
            const uint32_t acc = taddr + 256u * x + lanes + (uint32_t)(16 * cpart);
            uint32_t r[4][16];
#pragma unroll
            for (int c = 0; c < 4; ++c) tc_ld_16cols_issue(acc + 64u * c, r[c]);
#pragma unroll
            for (int c = 0; c < 4; ++c) tc_ld_wait16(r[c]);
            const float2 *bv2 = reinterpret_cast<const float2 *>(bv);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t *rc = r[c];
                const int col0 = 64 * c + 16 * cpart;
                uint32_t w[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const float2 y = silu_pair(make_float2(__uint_as_float(rc[2 * t]), __uint_as_float(rc[2 * t + 1])),
                                               bv2[col0 / 2 + t]);
                    w[t] = cvt_bf16x2(y.x, y.y);
                }
                unsigned char *blk = H + c * 16384;
                *reinterpret_cast<uint4 *>(blk + sw128_offset(row, 16 * cpart)) = make_uint4(w[0], w[1], w[2], w[3]);
                *reinterpret_cast<uint4 *>(blk + sw128_offset(row, 16 * cpart + 8)) =
                    make_uint4(w[4], w[5], w[6], w[7]);
                fence_proxy_async_smem();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&chunk[4 * x + c]);
            }
            return true;
        };
        // head of tile x (tile index t): logit = sum_c BF16(SiLU(z3 + b3)) w4 + b4.
        // Every warp writes its partial sums and arrives on partd[x]; warps
        // 0-3 (one row each, threads 0..127) wait for them and write the
        // logits; every warp then puts its share of the next pair's features
        // of this slot (tile tn) into K-block 0.  The feature arrival comes
        // last: the next layer-1 MMAs (which overwrite the accumulator) and
        // the epilogues after them (which overwrite K-block 1, the partial
        // sums) wait for it.
        auto head = [&](int x, long long t, bool next, long long tn) {
            if (!(ok && mbar_wait_warp(&accr[x], nacc[x] & 1))) return false;
            ++nacc[x];
            tc_fence_after();
            unsigned char *H = x ? sH1 : sH0;
            float *part = reinterpret_cast<float *>(H + 16384);   // [4][128] in K-block 1
            const uint32_t acc = taddr + 256u * x + lanes + (uint32_t)(16 * cpart);
            uint32_t r[4][16];
#pragma unroll
            for (int c = 0; c < 4; ++c) tc_ld_16cols_issue(acc + 64u * c, r[c]);
#pragma unroll
            for (int c = 0; c < 4; ++c) tc_ld_wait16(r[c]);
            const float2 *b3 = reinterpret_cast<const float2 *>(bias.b3);
            const float2 *w4 = reinterpret_cast<const float2 *>(bias.w4);
            float2 sum = make_float2(0.f, 0.f);   // even and odd columns
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t *rc = r[c];
                const int col0 = 64 * c + 16 * cpart;
#pragma unroll
                for (int t2 = 0; t2 < 8; ++t2) {
                    const float2 y = silu_pair(make_float2(__uint_as_float(rc[2 * t2]), __uint_as_float(rc[2 * t2 + 1])),
                                               b3[col0 / 2 + t2]);
                    const uint32_t hb = cvt_bf16x2(y.x, y.y);   // the activations rounded to BF16
                    sum = fma2(make_float2(__uint_as_float(hb << 16), __uint_as_float(hb & 0xFFFF0000u)),
                               w4[col0 / 2 + t2], sum);
                }
            }
            part[cpart * 128 + row] = sum.x + sum.y;
            __syncwarp();
            if (lane == 0) mbar_arrive(&partd[x]);
            bool good = true;
            if (warp < 4) {
                good = mbar_wait_warp(&partd[x], npart[x] & 1);
                if (good && t * 128 + tid < real)
                    logit[t * 128 + tid] = ((part[tid] + part[128 + tid]) + (part[256 + tid] + part[384 + tid])) + bias.b4;
            }
            ++npart[x];
            if (good && next) features(tn, H);
            fence_proxy_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0 && good) mbar_arrive(&feat[x]);
            return good;
        };
        for (long long p = blockIdx.x; p < npairs; p += gridDim.x) {
            const long long pn = p + gridDim.x;
            const bool next = pn < npairs;
            ok = epilogue(0, bias.b1);
            ok = epilogue(1, bias.b1);
            ok = epilogue(0, bias.b2);
            ok = epilogue(1, bias.b2);
            ok = head(0, 2 * p, next, 2 * pn);
            ok = head(1, 2 * p + 1, next, 2 * pn + 1);
            if (!ok) break;   // (each warp on its own: no CTA-wide barrier in the loop)
        }
    }
    if (!ok && lane == 0) atomicExch(err, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(taddr, 512);
}

}  // namespace ens

using namespace ens;

// ---------------------------------------------------------------------------
// surrogate object
// ---------------------------------------------------------------------------
struct ens_surrogate {
    cudaStream_t s = nullptr;
    ParamLayout L{};
    float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W3b = nullptr, *W2t = nullptr, *W3t = nullptr;
    int *err = nullptr;
    long long steps = 0;
    // work buffers for a given padded row count
    long long cap = 0;
    __nv_bfloat16 *X = nullptr, *Xt = nullptr, *H1 = nullptr, *H2 = nullptr, *H3 = nullptr, *H1t = nullptr,
                  *H2t = nullptr, *dZ = nullptr, *dZt = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr, *logit = nullptr, *dlogit = nullptr, *q = nullptr,
          *target = nullptr, *dH = nullptr, *part = nullptr;
    double *lam = nullptr, *loss = nullptr, *wq = nullptr, *pdf = nullptr;
    uint32_t *lam5 = nullptr;   // BF16 of lambda / 5 per lambda value (fused inference)
    int groups_cap = 0;
    unsigned char *img = nullptr;   // swizzled W1 | W2 | W3 images for the fused inference kernel
    int sms = 0;
};

namespace {

constexpr int kMaxSplit = 32;

bool alloc_work(ens_surrogate *S, long long rows, int groups)
{
    if (rows <= S->cap && groups <= S->groups_cap) return true;
    auto fr = [&](void *p) { if (p) cudaFree(p); };
    for (void *p : {(void *)S->X, (void *)S->Xt, (void *)S->H1, (void *)S->H2, (void *)S->H3, (void *)S->H1t,
                    (void *)S->H2t, (void *)S->dZ, (void *)S->dZt, (void *)S->Z1, (void *)S->Z2, (void *)S->Z3,
                    (void *)S->logit, (void *)S->dlogit, (void *)S->q, (void *)S->target, (void *)S->dH,
                    (void *)S->part, (void *)S->lam, (void *)S->lam5, (void *)S->loss})
        fr(p);
    bool ok = true;
    auto al = [&](auto **p, size_t bytes) {
        if (cudaMalloc((void **)p, bytes) != cudaSuccess) ok = false;
    };
    const size_t bh = sizeof(__nv_bfloat16) * rows * kHid;
    al(&S->X, sizeof(__nv_bfloat16) * rows * kIn);
    al(&S->Xt, sizeof(__nv_bfloat16) * rows * kIn);
    al(&S->H1, bh); al(&S->H2, bh); al(&S->H3, bh); al(&S->H1t, bh); al(&S->H2t, bh);
    al(&S->dZ, bh); al(&S->dZt, bh);
    const size_t fz = sizeof(float) * rows * kHid;
    al(&S->Z1, fz); al(&S->Z2, fz); al(&S->Z3, fz); al(&S->dH, fz);
    al(&S->logit, sizeof(float) * rows);
    al(&S->dlogit, sizeof(float) * rows);
    al(&S->q, sizeof(float) * rows);
    al(&S->target, sizeof(float) * rows);
    al(&S->part, sizeof(float) * kMaxSplit * kHid * kHid);
    al(&S->lam, sizeof(double) * 4096);
    al(&S->lam5, sizeof(uint32_t) * 4096);
    al(&S->loss, sizeof(double) * (groups + 1));
    S->cap = ok ? rows : 0;
    S->groups_cap = ok ? groups : 0;
    return ok;
}

int blocks(long long n, int t) { return (int)((n + t - 1) / t); }

// forward through the network for `rows` padded rows of features in S->X
bool forward(ens_surrogate *S, long long rows, bool keep_t)
{
    cudaStream_t s = S->s;
    const ParamLayout &L = S->L;
    if (!gemm(S->X, kIn, S->W1b, kIn, S->Z1, kHid, (int)rows, kHid, kIn, 1, S->err, s)) return false;
    k_bias_silu<<<blocks(rows * kHid, 256), 256, 0, s>>>(S->Z1, S->p + L.b1, rows, S->H1, keep_t ? S->H1t : nullptr);
    if (!gemm(S->H1, kHid, S->W2b, kHid, S->Z2, kHid, (int)rows, kHid, kHid, 1, S->err, s)) return false;
    k_bias_silu<<<blocks(rows * kHid, 256), 256, 0, s>>>(S->Z2, S->p + L.b2, rows, S->H2, keep_t ? S->H2t : nullptr);
    if (!gemm(S->H2, kHid, S->W3b, kHid, S->Z3, kHid, (int)rows, kHid, kHid, 1, S->err, s)) return false;
    k_bias_silu<<<blocks(rows * kHid, 256), 256, 0, s>>>(S->Z3, S->p + L.b3, rows, S->H3, nullptr);
    k_head<<<blocks(rows * 32, 256), 256, 0, s>>>(S->H3, S->p + L.w4, S->p + L.b4, rows, S->logit);
    return true;
}

// biases and head of the current parameters (host copy for the kernel parameters)
// the fused kernel takes b / 2 for the hidden layers (exact in FP32)
bool halve_biases(MlpBias *b)
{
    for (int i = 0; i < kHid; ++i) {
        b->b1[i] *= 0.5f;
        b->b2[i] *= 0.5f;
        b->b3[i] *= 0.5f;
    }
    return true;
}

bool mlp_bias(ens_surrogate *S, MlpBias *b)
{
    const ParamLayout &L = S->L;
    cudaStream_t s = S->s;
    return cudaMemcpyAsync(b->b1, S->p + L.b1, sizeof(float) * kHid, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
           cudaMemcpyAsync(b->b2, S->p + L.b2, sizeof(float) * kHid, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
           cudaMemcpyAsync(b->b3, S->p + L.b3, sizeof(float) * kHid, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
           cudaMemcpyAsync(b->w4, S->p + L.w4, sizeof(float) * kHid, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
           cudaMemcpyAsync(&b->b4, S->p + L.b4, sizeof(float), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
           cudaStreamSynchronize(s) == cudaSuccess && halve_biases(b);
}

// the fused inference kernel over `real` rows of the feature table ftab
// (one CTA per tile pair, at most one per SM)
void launch_infer(ens_surrogate *S, const RowSpec &rs, const uint4 *ftab, long long real, const MlpBias &bias)
{
    const long long ntiles = (real + 127) / 128;
    const int grid = (int)std::min<long long>((ntiles + 1) / 2, S->sms > 0 ? S->sms : 1);
    unsigned char *i1 = S->img, *i2 = S->img + 32768, *i3 = S->img + 32768 + 131072;
    k_mlp_infer_pair<<<grid, kPairThreads, kPairSmem, S->s>>>(rs, ftab, S->lam5, real, ntiles, i1, i2, i3, bias,
                                                              S->logit, S->err);
}

// fused inference of `real` rows (lambda values in S->lam) into S->logit
bool forward_fused(ens_surrogate *S, const RowSpec &rs, long long real)
{
    cudaStream_t s = S->s;
    const long long n = (long long)kHid * kHid;
    MlpBias bias;
    if (!mlp_bias(S, &bias)) return false;
    k_pack_weights_img<<<blocks(n, 256), 256, 0, s>>>(S->p, S->img, S->img + 32768, S->img + 32768 + 131072);
    const int nlam = (int)(real / rs.per_member);
    uint4 *ftab = reinterpret_cast<uint4 *>(S->Xt);   // the training path's transposed features: free here
    k_feature_table<<<blocks(std::max(rs.per_member, nlam), 256), 256, 0, s>>>(rs, S->lam, nlam, ftab, S->lam5);
    launch_infer(S, rs, ftab, real, bias);
    return cudaGetLastError() == cudaSuccess;
}

int pick_split(long long rows)
{
    int sp = kMaxSplit;
    while (sp > 1 && (rows % (64LL * sp) != 0 || rows / sp < 512)) --sp;
    return sp;
}

// backward pass into S->g (gradients of the mean group loss)
bool backward(ens_surrogate *S, long long rows, long long real)
{
    cudaStream_t s = S->s;
    const ParamLayout &L = S->L;
    k_head_grad<<<kHid + 1, 256, 0, s>>>(S->dlogit, S->H3, real, S->g + L.w4, S->g + L.b4);
    k_head_back<<<blocks(rows * kHid, 256), 256, 0, s>>>(S->dlogit, S->p + L.w4, S->Z3, rows, real, S->dZ, S->dZt);
    const int sp = pick_split(rows);
    // layer 3: dW3 = dZ3^T H2, db3, dH2 = dZ3 W3
    if (!gemm(S->dZt, (int)rows, S->H2t, (int)rows, S->part, kHid, kHid, kHid, (int)rows, sp, S->err, s)) return false;
    k_sum_splits<<<blocks((long long)kHid * kHid, 256), 256, 0, s>>>(S->part, sp, (long long)kHid * kHid, S->g + L.W3);
    k_colsum_bf16<<<kHid, 256, 0, s>>>(S->dZ, rows, S->g + L.b3);
    if (!gemm(S->dZ, kHid, S->W3t, kHid, S->dH, kHid, (int)rows, kHid, kHid, 1, S->err, s)) return false;
    k_silu_back<<<blocks(rows * kHid, 256), 256, 0, s>>>(S->dH, S->Z2, rows, S->dZ, S->dZt);
    // layer 2
    if (!gemm(S->dZt, (int)rows, S->H1t, (int)rows, S->part, kHid, kHid, kHid, (int)rows, sp, S->err, s)) return false;
    k_sum_splits<<<blocks((long long)kHid * kHid, 256), 256, 0, s>>>(S->part, sp, (long long)kHid * kHid, S->g + L.W2);
    k_colsum_bf16<<<kHid, 256, 0, s>>>(S->dZ, rows, S->g + L.b2);
    if (!gemm(S->dZ, kHid, S->W2t, kHid, S->dH, kHid, (int)rows, kHid, kHid, 1, S->err, s)) return false;
    k_silu_back<<<blocks(rows * kHid, 256), 256, 0, s>>>(S->dH, S->Z1, rows, S->dZ, S->dZt);
    // layer 1: dW1 = dZ1^T X (N = 64)
    if (!gemm(S->dZt, (int)rows, S->Xt, (int)rows, S->part, kIn, kHid, kIn, (int)rows, sp, S->err, s)) return false;
    k_sum_splits<<<blocks((long long)kHid * kIn, 256), 256, 0, s>>>(S->part, sp, (long long)kHid * kIn, S->g + L.W1);
    k_colsum_bf16<<<kHid, 256, 0, s>>>(S->dZ, rows, S->g + L.b1);
    return true;
}

long long pad128(long long r) { return (r + 127) / 128 * 128; }

// targets: normalised in-range histograms of each member and kind
void make_targets(int n, const uint64_t *counts, const ens_hist_spec *h, std::vector<float> &t)
{
    const int nq = h->qr_bins, nt = h->tail_bins;
    const int per = nq * nq + 2 * nt;
    const long long L = counts_len_of(nq, nt, h->grad_bins);
    t.assign((size_t)n * per, 0.f);
    for (int i = 0; i < n; ++i) {
        const uint64_t *c = counts + (size_t)i * L;
        const int off[3] = {0, nq * nq, nq * nq + nt};
        const int len[3] = {nq * nq, nt, nt};
        for (int k = 0; k < 3; ++k) {
            double s = 0.0;
            for (int b = 0; b < len[k]; ++b) s += (double)c[off[k] + b];
            for (int b = 0; b < len[k]; ++b)
                t[(size_t)i * per + off[k] + b] = s > 0.0 ? (float)((double)c[off[k] + b] / s) : 0.f;
        }
    }
}

}  // namespace

extern "C" {

ens_status ens_surrogate_create(uint64_t seed, void *stream, ens_surrogate **out)
{
    if (!out) return ENS_EINVAL;
    *out = nullptr;
    ens_surrogate *S = new ens_surrogate();
    S->s = (cudaStream_t)stream;
    S->L = param_layout();
    const long long n = S->L.total;
    bool ok = gemm_prepare() == cudaSuccess;
    ok = ok && cudaMalloc(&S->p, sizeof(float) * n) == cudaSuccess && cudaMalloc(&S->g, sizeof(float) * n) == cudaSuccess &&
         cudaMalloc(&S->m1, sizeof(float) * n) == cudaSuccess && cudaMalloc(&S->m2, sizeof(float) * n) == cudaSuccess &&
         cudaMalloc(&S->W1b, sizeof(__nv_bfloat16) * kHid * kIn) == cudaSuccess &&
         cudaMalloc(&S->W2b, sizeof(__nv_bfloat16) * kHid * kHid) == cudaSuccess &&
         cudaMalloc(&S->W3b, sizeof(__nv_bfloat16) * kHid * kHid) == cudaSuccess &&
         cudaMalloc(&S->W2t, sizeof(__nv_bfloat16) * kHid * kHid) == cudaSuccess &&
         cudaMalloc(&S->W3t, sizeof(__nv_bfloat16) * kHid * kHid) == cudaSuccess &&
         cudaMalloc(&S->err, sizeof(int)) == cudaSuccess && cudaMalloc(&S->wq, sizeof(double) * 4096) == cudaSuccess &&
         cudaMalloc(&S->pdf, sizeof(double) * 1 << 20) == cudaSuccess &&
         cudaMalloc(&S->img, 32768 + 2 * 131072) == cudaSuccess &&
         cudaFuncSetAttribute(k_mlp_infer_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPairSmem) ==
             cudaSuccess;
    int dev = 0;
    ok = ok && cudaGetDevice(&dev) == cudaSuccess &&
         cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
    if (!ok) {
        delete S;
        return ENS_ENOMEM;
    }
    cudaMemsetAsync(S->err, 0, sizeof(int), S->s);
    cudaMemsetAsync(S->m1, 0, sizeof(float) * n, S->s);
    cudaMemsetAsync(S->m2, 0, sizeof(float) * n, S->s);
    k_init_params<<<blocks(n, 256), 256, 0, S->s>>>(S->p, n, seed);
    k_pack_weights<<<blocks((long long)kHid * kHid, 256), 256, 0, S->s>>>(S->p, S->W1b, S->W2b, S->W3b, S->W2t, S->W3t);
    if (cudaStreamSynchronize(S->s) != cudaSuccess) {
        delete S;
        return ENS_ECUDA;
    }
    *out = S;
    return ENS_OK;
}

ens_status ens_surrogate_destroy(ens_surrogate *S)
{
    if (!S) return ENS_EINVAL;
    cudaStreamSynchronize(S->s);
    for (void *p : {(void *)S->p, (void *)S->g, (void *)S->m1, (void *)S->m2, (void *)S->W1b, (void *)S->W2b,
                    (void *)S->W3b, (void *)S->W2t, (void *)S->W3t, (void *)S->err, (void *)S->wq, (void *)S->pdf,
                    (void *)S->img,
                    (void *)S->X, (void *)S->Xt, (void *)S->H1, (void *)S->H2, (void *)S->H3, (void *)S->H1t,
                    (void *)S->H2t, (void *)S->dZ, (void *)S->dZt, (void *)S->Z1, (void *)S->Z2, (void *)S->Z3,
                    (void *)S->logit, (void *)S->dlogit, (void *)S->q, (void *)S->target, (void *)S->dH,
                    (void *)S->part, (void *)S->lam, (void *)S->lam5, (void *)S->loss})
        if (p) cudaFree(p);
    delete S;
    return ENS_OK;
}

size_t ens_surrogate_param_count(void) { return (size_t)param_layout().total; }

ens_status ens_surrogate_get_params(ens_surrogate *S, float *host)
{
    if (!S || !host) return ENS_EINVAL;
    if (cudaMemcpyAsync(host, S->p, sizeof(float) * S->L.total, cudaMemcpyDeviceToHost, S->s) != cudaSuccess ||
        cudaStreamSynchronize(S->s) != cudaSuccess)
        return ENS_ECUDA;
    return ENS_OK;
}

ens_status ens_surrogate_set_params(ens_surrogate *S, const float *host)
{
    if (!S || !host) return ENS_EINVAL;
    if (cudaMemcpyAsync(S->p, host, sizeof(float) * S->L.total, cudaMemcpyHostToDevice, S->s) != cudaSuccess)
        return ENS_ECUDA;
    k_pack_weights<<<blocks((long long)kHid * kHid, 256), 256, 0, S->s>>>(S->p, S->W1b, S->W2b, S->W3b, S->W2t, S->W3t);
    if (cudaStreamSynchronize(S->s) != cudaSuccess) return ENS_ECUDA;
    return ENS_OK;
}

static ens_status load_batch(ens_surrogate *S, int n, const double *lambdas, const uint64_t *counts,
                             const ens_hist_spec *h, long long *rows_pad, long long *real, RowSpec *rs)
{
    if (!S || n <= 0 || n > 4096 || !lambdas || !h || h->qr_bins < 1 || h->tail_bins < 1) return ENS_EINVAL;
    rs->nq = h->qr_bins;
    rs->nt = h->tail_bins;
    rs->per_member = h->qr_bins * h->qr_bins + 2 * h->tail_bins;
    *real = (long long)n * rs->per_member;
    *rows_pad = pad128(*real);
    if (*rows_pad % 64 != 0) return ENS_EINVAL;
    if (!alloc_work(S, *rows_pad, 3 * n)) return ENS_ENOMEM;
    if (cudaMemcpyAsync(S->lam, lambdas, sizeof(double) * n, cudaMemcpyHostToDevice, S->s) != cudaSuccess)
        return ENS_ECUDA;
    k_features<<<blocks(*rows_pad, 256), 256, 0, S->s>>>(*rs, S->lam, n, *rows_pad, S->X, S->Xt);
    if (counts) {
        std::vector<float> t;
        make_targets(n, counts, h, t);
        if (cudaMemcpyAsync(S->target, t.data(), sizeof(float) * t.size(), cudaMemcpyHostToDevice, S->s) !=
            cudaSuccess ||
            cudaStreamSynchronize(S->s) != cudaSuccess)
            return ENS_ECUDA;
    }
    return ENS_OK;
}

static ens_status check_err(ens_surrogate *S)
{
    int e = 0;
    if (cudaMemcpyAsync(&e, S->err, sizeof(int), cudaMemcpyDeviceToHost, S->s) != cudaSuccess ||
        cudaStreamSynchronize(S->s) != cudaSuccess)
        return ENS_ECUDA;
    return e ? ENS_ETIMEOUT : ENS_OK;
}

ens_status ens_surrogate_loss_grad(ens_surrogate *S, int n, const double *lambdas, const uint64_t *counts,
                                   const ens_hist_spec *h, double *loss, float *grad_host)
{
    long long rows, real;
    RowSpec rs;
    if (!counts) return ENS_EINVAL;
    ens_status st = load_batch(S, n, lambdas, counts, h, &rows, &real, &rs);
    if (st != ENS_OK) return st;
    const double wgt = 1.0 / (3.0 * n);
    if (!forward(S, rows, true)) return ENS_EINVAL;
    cudaMemsetAsync(S->dlogit, 0, sizeof(float) * rows, S->s);
    k_softmax_ce<<<3 * n, 256, 0, S->s>>>(S->logit, S->target, rs.nq, rs.nt, wgt, S->q, S->dlogit, S->loss);
    if (!backward(S, rows, real)) return ENS_EINVAL;
    if (cudaGetLastError() != cudaSuccess) return ENS_ECUDA;
    std::vector<double> lp(3 * n);
    if (cudaMemcpyAsync(lp.data(), S->loss, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, S->s) != cudaSuccess)
        return ENS_ECUDA;
    if (grad_host &&
        cudaMemcpyAsync(grad_host, S->g, sizeof(float) * S->L.total, cudaMemcpyDeviceToHost, S->s) != cudaSuccess)
        return ENS_ECUDA;
    st = check_err(S);
    if (st != ENS_OK) return st;
    if (loss) {
        double t = 0.0;
        for (double v : lp) t += v;
        *loss = t;
    }
    return ENS_OK;
}

ens_status ens_surrogate_train(ens_surrogate *S, int n, const double *lambdas, const uint64_t *counts,
                               const ens_hist_spec *h, int steps, double lr, double *final_loss)
{
    long long rows, real;
    RowSpec rs;
    if (!counts || steps < 0 || !(lr > 0.0)) return ENS_EINVAL;
    ens_status st = load_batch(S, n, lambdas, counts, h, &rows, &real, &rs);
    if (st != ENS_OK) return st;
    const double wgt = 1.0 / (3.0 * n);
    const long long np = S->L.total;
    for (int it = 0; it < steps; ++it) {
        if (!forward(S, rows, true)) return ENS_EINVAL;
        k_softmax_ce<<<3 * n, 256, 0, S->s>>>(S->logit, S->target, rs.nq, rs.nt, wgt, nullptr, S->dlogit,
                                             it == steps - 1 ? S->loss : nullptr);
        if (!backward(S, rows, real)) return ENS_EINVAL;
        S->steps += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float bc1 = 1.f - powf(b1, (float)S->steps), bc2 = 1.f - powf(b2, (float)S->steps);
        // cosine decay over the call's steps, from lr to lr / 20
        const double lr_t = lr * (0.05 + 0.95 * 0.5 * (1.0 + std::cos(3.14159265358979323846 * it / steps)));
        k_adam<<<blocks(np, 256), 256, 0, S->s>>>(S->p, S->g, S->m1, S->m2, np, (float)lr_t, b1, b2, 1e-8f, bc1, bc2);
        k_pack_weights<<<blocks((long long)kHid * kHid, 256), 256, 0, S->s>>>(S->p, S->W1b, S->W2b, S->W3b, S->W2t,
                                                                             S->W3t);
    }
    if (cudaGetLastError() != cudaSuccess) return ENS_ECUDA;
    st = check_err(S);
    if (st != ENS_OK) return st;
    if (final_loss && steps > 0) {
        std::vector<double> lp(3 * n);
        if (cudaMemcpyAsync(lp.data(), S->loss, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, S->s) != cudaSuccess ||
            cudaStreamSynchronize(S->s) != cudaSuccess)
            return ENS_ECUDA;
        double t = 0.0;
        for (double v : lp) t += v;
        *final_loss = t;
    }
    return ENS_OK;
}

ens_status ens_surrogate_density(ens_surrogate *S, int n, const double *lambdas, const ens_hist_spec *h,
                                 double *probs)
{
    long long rows, real;
    RowSpec rs;
    ens_status st = load_batch(S, n, lambdas, nullptr, h, &rows, &real, &rs);
    if (st != ENS_OK) return st;
    if (!forward_fused(S, rs, real)) return ENS_ECUDA;
    k_softmax_ce<<<3 * n, 256, 0, S->s>>>(S->logit, nullptr, rs.nq, rs.nt, 1.0, S->q, nullptr, nullptr);
    if (cudaGetLastError() != cudaSuccess) return ENS_ECUDA;
    std::vector<float> q((size_t)real);
    if (cudaMemcpyAsync(q.data(), S->q, sizeof(float) * real, cudaMemcpyDeviceToHost, S->s) != cudaSuccess)
        return ENS_ECUDA;
    st = check_err(S);
    if (st != ENS_OK) return st;
    for (long long i = 0; i < real; ++i) probs[i] = q[i];
    return ENS_OK;
}

ens_status ens_surrogate_mixture(ens_surrogate *S, const ens_hist_spec *h, const ens_weight_spec *w, double lam_lo,
                                 double lam_hi, int nquad, ens_mixture_out *out)
{
    if (!S || !h || !w || !out || nquad < 1 || nquad > 4096 || !(lam_hi > lam_lo)) return ENS_EINVAL;
    if (w->kind != ENS_W_GAUSS_PAPER && w->kind != ENS_W_GAUSS) return ENS_EINVAL;
    RowSpec rs{h->qr_bins, h->tail_bins, h->qr_bins * h->qr_bins + 2 * h->tail_bins};
    const long long real = (long long)nquad * rs.per_member, rows = pad128(real);
    if (rs.per_member > (1 << 20)) return ENS_EINVAL;
    if (!alloc_work(S, rows, 3 * nquad)) return ENS_ENOMEM;
    k_quad_weights<<<1, 256, 0, S->s>>>(lam_lo, lam_hi, nquad, w->kind, w->c, w->Z, w->mu, w->sigma, S->lam, S->wq);
    if (!forward_fused(S, rs, real)) return ENS_ECUDA;
    k_softmax_ce<<<3 * nquad, 256, 0, S->s>>>(S->logit, nullptr, rs.nq, rs.nt, 1.0, S->q, nullptr, nullptr);
    const double dq = 2.0 * h->q_lim / h->qr_bins, dr = 2.0 * h->r_lim / h->qr_bins;
    const double dt = (h->tail_hi - h->tail_lo) / h->tail_bins;
    k_quad_mix<<<blocks(rs.per_member, 256), 256, 0, S->s>>>(S->q, S->wq, nquad, rs.per_member, rs.nq, dq, dr, dt,
                                                             S->pdf);
    if (cudaGetLastError() != cudaSuccess) return ENS_ECUDA;
    std::vector<double> pdf(rs.per_member);
    if (cudaMemcpyAsync(pdf.data(), S->pdf, sizeof(double) * rs.per_member, cudaMemcpyDeviceToHost, S->s) !=
        cudaSuccess)
        return ENS_ECUDA;
    ens_status st = check_err(S);
    if (st != ENS_OK) return st;
    const int nq2 = rs.nq * rs.nq;
    if (out->pdf_qr) std::memcpy(out->pdf_qr, pdf.data(), sizeof(double) * nq2);
    if (out->pdf_eps) std::memcpy(out->pdf_eps, pdf.data() + nq2, sizeof(double) * rs.nt);
    if (out->pdf_ens) std::memcpy(out->pdf_ens, pdf.data() + nq2 + rs.nt, sizeof(double) * rs.nt);
    out->covered = 1.0;
    return ENS_OK;
}

// average time of the hidden-layer GEMM (rows x 256 x 256) on the object's
// buffers, CUDA events on its stream (profiling)
ens_status ens_surrogate_time_gemm(ens_surrogate *S, long long rows, int iters, double *ms)
{
    if (!S || rows <= 0 || iters < 1 || !ms) return ENS_EINVAL;
    rows = pad128(rows);
    if (!alloc_work(S, rows, 3)) return ENS_ENOMEM;
    cudaMemsetAsync(S->H1, 0, sizeof(__nv_bfloat16) * rows * kHid, S->s);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    gemm(S->H1, kHid, S->W2b, kHid, S->Z2, kHid, (int)rows, kHid, kHid, 1, S->err, S->s);   // warm-up
    cudaEventRecord(a, S->s);
    for (int i = 0; i < iters; ++i) gemm(S->H1, kHid, S->W2b, kHid, S->Z2, kHid, (int)rows, kHid, kHid, 1, S->err, S->s);
    cudaEventRecord(b, S->s);
    float t = 0.f;
    const cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return ENS_ECUDA;
    *ms = t / iters;
    return check_err(S);
}

// logits of the network at n lambda values, by the fused inference kernel
// (fused != 0) or by the layer-by-layer training forward pass (tests)
ens_status ens_surrogate_logits(ens_surrogate *S, int n, const double *lambdas, const ens_hist_spec *h, int fused,
                                float *logits)
{
    long long rows, real;
    RowSpec rs;
    if (!logits) return ENS_EINVAL;
    ens_status st = load_batch(S, n, lambdas, nullptr, h, &rows, &real, &rs);
    if (st != ENS_OK) return st;
    if (fused ? !forward_fused(S, rs, real) : !forward(S, rows, false)) return ENS_ECUDA;
    if (cudaMemcpyAsync(logits, S->logit, sizeof(float) * real, cudaMemcpyDeviceToHost, S->s) != cudaSuccess)
        return ENS_ECUDA;
    return check_err(S);
}

// average time of the fused inference kernel over nquad lambda values of a
// histogram layout, CUDA events on the object's stream (profiling)
ens_status ens_surrogate_time_infer(ens_surrogate *S, const ens_hist_spec *h, int nquad, int iters, double *ms)
{
    if (!S || !h || nquad < 1 || nquad > 4096 || iters < 1 || !ms) return ENS_EINVAL;
    RowSpec rs{h->qr_bins, h->tail_bins, h->qr_bins * h->qr_bins + 2 * h->tail_bins};
    const long long real = (long long)nquad * rs.per_member, rows = pad128(real);
    if (!alloc_work(S, rows, 3 * nquad)) return ENS_ENOMEM;
    k_quad_weights<<<1, 256, 0, S->s>>>(-5.0, 5.0, nquad, 1, 0.0, 0.0, 0.0, 1.0, S->lam, S->wq);
    k_pack_weights_img<<<blocks((long long)kHid * kHid, 256), 256, 0, S->s>>>(S->p, S->img, S->img + 32768,
                                                                              S->img + 32768 + 131072);
    MlpBias bias;
    if (!mlp_bias(S, &bias)) return ENS_ECUDA;
    uint4 *ftab = reinterpret_cast<uint4 *>(S->Xt);
    k_feature_table<<<blocks(std::max(rs.per_member, nquad), 256), 256, 0, S->s>>>(rs, S->lam, nquad, ftab, S->lam5);
    auto launch = [&]() { launch_infer(S, rs, ftab, real, bias); };
    launch();   // warm-up
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, S->s);
    for (int i = 0; i < iters; ++i) launch();
    cudaEventRecord(b, S->s);
    float t = 0.f;
    const cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return ENS_ECUDA;
    *ms = t / iters;
    return check_err(S);
}

// tensor-core GEMM check: C = A B^T for host BF16 bit patterns (tests)
ens_status ens_tc_gemm_check(const uint16_t *A, const uint16_t *B, float *C, int M, int N, int K, int ksplit)
{
    if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || ksplit < 1 || ksplit > kMaxSplit) return ENS_EINVAL;
    if (M % 128 || K % (64 * ksplit) || N % 64) return ENS_EINVAL;
    if (gemm_prepare() != cudaSuccess) return ENS_ECUDA;
    void *dA = nullptr, *dB = nullptr, *dC = nullptr, *dE = nullptr;
    ens_status st = ENS_OK;
    if (cudaMalloc(&dA, sizeof(uint16_t) * M * K) != cudaSuccess || cudaMalloc(&dB, sizeof(uint16_t) * N * K) != cudaSuccess ||
        cudaMalloc(&dC, sizeof(float) * M * N * ksplit) != cudaSuccess || cudaMalloc(&dE, sizeof(int)) != cudaSuccess)
        st = ENS_ENOMEM;
    if (st == ENS_OK) {
        cudaMemcpy(dA, A, sizeof(uint16_t) * M * K, cudaMemcpyHostToDevice);
        cudaMemcpy(dB, B, sizeof(uint16_t) * N * K, cudaMemcpyHostToDevice);
        cudaMemset(dE, 0, sizeof(int));
        gemm((const __nv_bfloat16 *)dA, K, (const __nv_bfloat16 *)dB, K, (float *)dC, N, M, N, K, ksplit, (int *)dE, 0);
        if (ksplit > 1) {
            k_sum_splits<<<blocks((long long)M * N, 256), 256>>>((const float *)dC, ksplit, (long long)M * N,
                                                                (float *)dC + (long long)M * N * (ksplit - 1));
        }
        int e = 0;
        if (cudaDeviceSynchronize() != cudaSuccess) st = ENS_ECUDA;
        cudaMemcpy(&e, dE, sizeof(int), cudaMemcpyDeviceToHost);
        if (e) st = ENS_ETIMEOUT;
        if (st == ENS_OK)
            cudaMemcpy(C, (float *)dC + (ksplit > 1 ? (long long)M * N * (ksplit - 1) : 0), sizeof(float) * M * N,
                       cudaMemcpyDeviceToHost);
    }
    for (void *p : {dA, dB, dC, dE})
        if (p) cudaFree(p);
    return st;
}

}  // extern "C"
