// Persistent stage kernel: every member of every grid size advances one RK
// stage in one launch (grid sizes 128, 256 and 384, the sizes of the
// uneven-size batch).
//
// One cooperative launch per stage, one 256-thread CTA per SM.  The host
// lays out the stage's work items in dependency order -- the inverse-x
// tiles of every member, then the inverse-y tiles, the z-pass row-group
// chunks, the forward-y tiles, the forward-x/update tiles, and one stage
// finish per member -- and each CTA takes the next item from a global
// counter.  An item of pass p of member m waits (bounded) until every item
// of pass p - 1 of that member is done (a per-member, per-pass counter), runs
// the same pass body as the separate kernels on its coordinates, and counts
// itself done.  Every item's dependencies come earlier in the list and every
// CTA is resident (cooperative launch), so the earliest unfinished item can
// always run: no deadlock.  A wait that gives up flags the member
// (ENS_ETIMEOUT) and raises an abort flag: from then on every item only
// counts itself done (flagging its member), so the launch drains at once.
//
// This translation unit is compiled with global loads cached in L2 only
// (-dlcm=cg): within one launch a CTA reads data that other CTAs wrote after
// it may have cached an earlier version of the same lines (buffer A holds
// the inverse-x output for the inverse-y items and, later in the same
// stage, the forward-y output for the forward-x items).
#include "ens_launch.h"
#include "ens_kernels.cuh"
#include "ens_persist.h"
#include "ens_znl.cuh"

#include <algorithm>
#include <vector>

namespace ens {
namespace {

constexpr int kThreads = 256;
constexpr int kDepPolls = 1 << 22;   // bounded dependency wait (x 128 ns sleeps: about half a second)

// the pass variants with 256 threads at each size: 16-column tiles, the
// 16-thread-per-line FFT plan (the second plan at N = 128), the default z
// warp plan, the fused forward-x/update pass
template <int N>
__host__ __device__ constexpr int col_var() { return N == 128 ? 1 : 0; }

template <int N>
__host__ __device__ constexpr long long z_groups() { return (long long)N * N / ZCfg<N, 0>::LPW; }   // row groups per member

template <int N>
constexpr size_t smem_need()
{
    constexpr size_t a = smem_x<N, 16>(), b = smem_cols<N, 16>(), c = ZCfg<N, 0>::smem_bytes();
    return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

constexpr size_t kSmem = std::max({smem_need<128>(), smem_need<256>(), smem_need<384>()});
static_assert(kSmem + 128 <= 227 * 1024, "one CTA's shared memory");

static_assert(ColCfg<128, 16, col_var<128>()>::threads == kThreads, "256-thread column passes at 128");
static_assert(ColCfg<256, 16, col_var<256>()>::threads == kThreads, "256-thread column passes at 256");
static_assert(ColCfg<384, 16, col_var<384>()>::threads == kThreads, "256-thread column passes at 384");

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int N>
__device__ __forceinline__ void run_item(int kind, const Geo &g, const PItem &it, const PStageArgs &a,
                                         unsigned char *sm)
{
    constexpr int VX = col_var<N>();
    float2 *smf = reinterpret_cast<float2 *>(sm);
    switch (kind) {
    case kPIX:
        for (int t = 0; t < it.count; ++t) {
            inv_x_body<N, 0, 16, VX>(g, a.stage > 0 ? 1 : 0, it.a + t, it.m, smf);
            __syncthreads();
        }
        break;
    case kPIY:
        for (int t = 0; t < it.count; ++t) {
            inv_y_body<N, 16, VX>(g, it.a + t, it.b, it.m, smf);
            __syncthreads();
        }
        break;
    case kPZ: {
        const long long f = (long long)it.m * z_groups<N>() + it.a;
        znl_body<N, 0, true>(g, a.md, a.stage, f, ZCfg<N, 0>::WPB, f + it.count, sm);
        break;
    }
    case kPFY:
        for (int t = 0; t < it.count; ++t) {
            fwd_y_body<N, 16, VX>(g, it.a + t, it.b, it.m, smf);
            __syncthreads();
        }
        break;
    case kPFX:
        for (int t = 0; t < it.count; ++t) {
            fwd_x_body<N, 0, 16, VX>(g, a.md, a.stage, a.last, it.a + t, it.m, smf);
            __syncthreads();
        }
        break;
    default:
        if (threadIdx.x < 32) finish_body(a.md, g.partial, g.partial_blocks, a.stage, a.last, 0, g.first + it.m,
                                          threadIdx.x);
        break;
    }
}

__global__ void __launch_bounds__(kThreads, 1) k_stage_persist(const __grid_constant__ PStageArgs a)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ int s_item;
    __shared__ bool s_skip;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(a.next, 1u);
        __syncthreads();
        const int idx = s_item;
        if (idx >= a.nitems) break;
        const PItem it = a.items[idx];
        const int kind = it.kind, slot = it.slot;
        const Geo &g = a.g[slot];
        const int gm = g.first + it.m;
        // after a wait that gave up anywhere, the remaining items only count
        // themselves done: the launch drains instead of waiting item by item
        if (threadIdx.x == 0) {
            s_skip = ld_acquire(a.abort) != 0u;
            if (!s_skip && kind > 0) {
                const unsigned *dep = a.done + (long long)gm * kPKinds + (kind - 1);
                const unsigned need = a.need[slot][kind - 1];
                int k = 0;
                for (; k < kDepPolls && ld_acquire(dep) < need; ++k) __nanosleep(128);
                if (k == kDepPolls) {
                    atomicOr(&a.md[gm].flags, kFlagTimeout);
                    atomicExch(a.abort, 1u);
                    s_skip = true;
                }
            }
        }
        __syncthreads();
        if (!s_skip) {
            // data written by other CTAs (generic proxy) is read below by bulk
            // copies (async proxy) in the z pass
            asm volatile("fence.proxy.async;" ::: "memory");
            switch (g.N) {
            case 128: run_item<128>(kind, g, it, a, smraw); break;
            case 256: run_item<256>(kind, g, it, a, smraw); break;
            default: run_item<384>(kind, g, it, a, smraw); break;
            }
        } else if (threadIdx.x == 0) {
            atomicOr(&a.md[gm].flags, kFlagTimeout);   // this item's work was not done
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(a.done + (long long)gm * kPKinds + kind, 1u);
        }
    }
}

}  // namespace

bool persist_size_supported(int N) { return N == 128 || N == 256 || N == 384; }

// Work items of one stage for the groups (ascending N), in dependency order;
// need[slot][kind]: items of each kind per member.
void persist_items(const std::vector<Geo> &groups, std::vector<PItem> &items, unsigned need[kPSlots][kPKinds])
{
    items.clear();
    for (int s = 0; s < kPSlots; ++s)
        for (int k = 0; k < kPKinds; ++k) need[s][k] = 0;
    constexpr int kColRun = 4;      // column tiles per item
    constexpr int kZChunk = 512;    // z-pass row groups per item
    auto lpw = [](int N) { return N == 128 ? ZCfg<128, 0>::LPW : N == 256 ? ZCfg<256, 0>::LPW : ZCfg<384, 0>::LPW; };
    for (int kind = 0; kind < kPKinds; ++kind) {
        // larger grids first within a pass: their items are the longest
        for (int s = (int)groups.size() - 1; s >= 0; --s) {
            const Geo &g = groups[s];
            const int state_tiles = g.NK * g.NZp / 16, mid_tiles = g.N * g.NZp / 16;
            const long long zg = (long long)g.N * g.N / lpw(g.N);
            unsigned per = 0;
            for (int m = 0; m < g.members; ++m) {
                auto cols = [&](int ntiles, int b) {
                    for (int t0 = 0; t0 < ntiles; t0 += kColRun) {
                        items.push_back(PItem{kind, s, m, t0, b, std::min(kColRun, ntiles - t0)});
                        if (m == 0) ++per;
                    }
                };
                switch (kind) {
                case kPIX: cols(state_tiles, 0); break;
                case kPIY: for (int f = 0; f < 6; ++f) cols(mid_tiles, f); break;
                case kPZ:
                    for (long long c0 = 0; c0 < zg; c0 += kZChunk) {
                        items.push_back(PItem{kind, s, m, (int)c0, 0, (int)std::min<long long>(kZChunk, zg - c0)});
                        if (m == 0) ++per;
                    }
                    break;
                case kPFY: for (int f = 0; f < 3; ++f) cols(mid_tiles, f); break;
                case kPFX: cols(state_tiles, 0); break;
                default:
                    items.push_back(PItem{kind, s, m, 0, 0, 1});
                    if (m == 0) ++per;
                    break;
                }
            }
            need[s][kind] = per;
        }
    }
}

cudaError_t persist_prepare()
{
    return cudaFuncSetAttribute(k_stage_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
}

int persist_ctas_per_sm()
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stage_persist, kThreads, kSmem) != cudaSuccess)
        return 0;
    return per_sm;
}

cudaError_t launch_stage_persist(const PStageArgs &a, int ctas, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_stage_persist, a);
}

}  // namespace ens
