// Pass launchers of one grid size N = ENS_N.  The build compiles this file
// once per supported N (-DENS_N=16 ... 512), so the heavy template
// instantiations of the FFT passes spread over parallel compiler jobs.
#include "ens_fxsplit.cuh"
#include "ens_fxws.cuh"
#include "ens_launch.h"
#include "ens_stats.cuh"
#include "ens_znl.cuh"

#include <cstdio>

#ifndef ENS_N
#error "compile with -DENS_N=<grid size>"
#endif

namespace ens {
namespace {

constexpr int N = ENS_N;

template <class K>
cudaError_t allow_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// the second x-pass plan exists for some sizes only (a template, so that the
// discarded branch is never instantiated)
template <int M>
cudaError_t prepare_variants()
{
    cudaError_t e = cudaSuccess;
    if constexpr (has_fx_ws<M>())
        e = cudaFuncSetAttribute(k_fwd_x_ws<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WsCfg<M>::smem());
    if constexpr (has_zplan_variant(M)) {
        if (ZCfg<M, 1>::smem_bytes() > 48 * 1024)
            e = cudaFuncSetAttribute(k_znl<M, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)ZCfg<M, 1>::smem_bytes());
    }
    if constexpr (has_plan_variant(M)) {
        auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
        chk(allow_smem(k_inv_x<M, 0, 16, 1>, smem_x<M, 16>()));
        chk(allow_smem(k_inv_x<M, 0, 8, 1>, smem_x<M, 8>()));
        chk(allow_smem(k_fwd_x<M, 0, 16, 1>, smem_x<M, 16>()));
        chk(allow_smem(k_fwd_x<M, 0, 8, 1>, smem_x<M, 8>()));
    }
    return e;
}

cudaError_t prepare(int nq, int nt, int ng)
{
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    chk(allow_smem(k_inv_x<N, 0, 16>, smem_x<N, 16>()));
    chk(allow_smem(k_inv_x<N, 0, 8>, smem_x<N, 8>()));
    chk(prepare_variants<N>());
    chk(allow_smem(k_fwd_x_fft<N, 16>, smem_cols<N, 16>()));
    chk(allow_smem(k_inv_x<N, 1, 16>, smem_x<N, 16>()));
    chk(allow_smem(k_inv_y<N, 16>, smem_cols<N, 16>()));
    chk(allow_smem(k_inv_y<N, 8>, smem_cols<N, 8>()));
    chk(allow_smem(k_inv_y_grad<N, 16>, smem_cols<N, 16>()));
    chk(allow_smem(k_inv_y_grad<N, 8>, smem_cols<N, 8>()));
    chk(allow_smem(k_fwd_y<N, 16>, smem_cols<N, 16>()));
    chk(allow_smem(k_fwd_y<N, 8>, smem_cols<N, 8>()));
    chk(allow_smem(k_fwd_x<N, 0, 16>, smem_x<N, 16>()));
    chk(allow_smem(k_fwd_x<N, 0, 8>, smem_x<N, 8>()));
    chk(allow_smem(k_fwd_x<N, 1, 16>, smem_x<N, 16>()));
    chk(allow_smem(k_fwd_x<N, 2, 16>, smem_x<N, 16>()));
    chk(allow_smem(k_fwd_x<N, 3, 16>, smem_x<N, 16>()));
    chk(allow_smem(k_z<N, 0>, smem_rows<N>()));
    chk(allow_smem(k_z<N, 1>, smem_rows<N>()));
    chk(allow_smem(k_z<N, 3>, smem_rows<N>()));
    chk(allow_smem(k_z<N, 4>, smem_rows<N>()));
    chk(allow_smem(k_z_stats<N>, smem_stats<N>(nq, nt, ng)));
    chk(allow_smem(k_znl<N>, ZCfg<N>::smem_bytes()));
    return e;
}

template <int M>
int znl_per_sm_t(int var)
{
    int per_sm = 0;
    if constexpr (has_zplan_variant(M)) {
        if (var == 1) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_znl<M, 1>, 256, ZCfg<M, 1>::smem_bytes()) !=
                cudaSuccess)
                return 0;
            return per_sm;
        }
    }
    if (var != 0) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_znl<M>, 256, ZCfg<M>::smem_bytes()) != cudaSuccess)
        return 0;
    return per_sm;
}

int znl_per_sm(int var) { return znl_per_sm_t<N>(var); }

template <int M>
void launch_znl_t(const Geo &g, MemberDev *md, int stage, cudaStream_t s)
{
    if constexpr (has_zplan_variant(M)) {
        if (g.z_mode == 2) {
            k_znl<M, 1><<<g.z_ctas, 256, ZCfg<M, 1>::smem_bytes(), s>>>(g, md, stage);
            return;
        }
    }
    k_znl<M><<<g.z_ctas, 256, ZCfg<M>::smem_bytes(), s>>>(g, md, stage);
}

template <int M>
void launch_fx_ws_t(const Geo &g, MemberDev *md, int stage, int last, cudaStream_t s)
{
    if constexpr (has_fx_ws<M>()) {
        const long long tiles = (long long)WsCfg<M>::TILES * g.members;
        const int grid = (int)(tiles < g.sms ? tiles : g.sms);
        k_fwd_x_ws<M><<<grid, 2 * WsCfg<M>::TH, WsCfg<M>::smem(), s>>>(g, md, stage, last);
    }
}

template <int T, int VAR = 0>
void launch_cols(Pass pass, int mode, const Geo &g, MemberDev *md, int stage, int last, int arg, cudaStream_t s)
{
    constexpr int TC = ColCfg<N, T, VAR>::threads;
    const dim3 grid_state(g.NK * g.NZp / T, g.members);
    const int col_tiles_mid = N * g.NZp / T;
    switch (pass) {
    case Pass::IX:
        if (mode == 0) k_inv_x<N, 0, T, VAR><<<grid_state, TC, smem_x<N, T>(), s>>>(g, arg);
        break;
    case Pass::IY:
        // arg = number of fields, mode = first field (kIYGrad: the gradient
        // components from the six x-pass fields)
        if (mode == kIYGrad) k_inv_y_grad<N, T><<<dim3(8, col_tiles_mid, g.members), TC, smem_cols<N, T>(), s>>>(g);
        else k_inv_y<N, T><<<dim3(col_tiles_mid, arg, g.members), TC, smem_cols<N, T>(), s>>>(g, mode);
        break;
    case Pass::FY:
        k_fwd_y<N, T><<<dim3(col_tiles_mid, 3, g.members), TC, smem_cols<N, T>(), s>>>(g);
        break;
    case Pass::FX:
        if (mode == 0) k_fwd_x<N, 0, T, VAR><<<grid_state, TC, smem_x<N, T>(), s>>>(g, md, stage, last);
        break;
    default: break;
    }
}

// stage passes along x: tile width and FFT plan from the group's tuning
template <int M>
void launch_x_t(Pass pass, int mode, const Geo &g, MemberDev *md, int stage, int last, int arg, cudaStream_t s)
{
    if constexpr (has_plan_variant(M)) {
        if (g.plan_x == 1) {
            if (g.tile_x == 8) launch_cols<8, 1>(pass, mode, g, md, stage, last, arg, s);
            else launch_cols<16, 1>(pass, mode, g, md, stage, last, arg, s);
            return;
        }
    }
    if (g.tile_x == 8) launch_cols<8>(pass, mode, g, md, stage, last, arg, s);
    else launch_cols<16>(pass, mode, g, md, stage, last, arg, s);
}

void launch_x(Pass pass, int mode, const Geo &g, MemberDev *md, int stage, int last, int arg, cudaStream_t s)
{
    launch_x_t<N>(pass, mode, g, md, stage, last, arg, s);
}

void launch(Pass pass, int mode, const Geo &g, MemberDev *md, const HistDev *h, int stage, int last, int arg,
            cudaStream_t s)
{
    // the kernels take the geometry from Dims<N>; a Geo built otherwise is a bug
    using D = Dims<N>;
    if (g.N != N || g.kc != D::KC || g.NK != D::NK || g.NZ != D::NZ || g.NZp != D::NZP || g.sU != D::SU ||
        g.sA != D::SA || g.sB != D::SB) {
        fprintf(stderr, "libens: geometry of N=%d does not match its compiled layout\n", N);
        return;
    }
    constexpr int RZ = RowCfg<N>::RZ;
    constexpr int TZ = RZ * RowCfg<N>::P;   // 256 threads, warp-local rows
    constexpr int TC = ColCfg<N, 16>::threads;
    const dim3 grid_state(g.NK * g.NZp / 16, g.members);
    switch (pass) {
    case Pass::IX:
        if (mode == 0) {
            launch_x(pass, mode, g, md, stage, last, arg, s);
        } else {
            k_inv_x<N, 1, 16><<<grid_state, TC, smem_x<N, 16>(), s>>>(g, arg);
        }
        break;
    case Pass::IY:
    case Pass::FY:
        if (g.tile_y == 8) launch_cols<8>(pass, mode, g, md, stage, last, arg, s);
        else launch_cols<16>(pass, mode, g, md, stage, last, arg, s);
        break;
    case Pass::Z: {
        const dim3 grid(N * N / RZ, g.members);
        switch (mode) {
        case 0:
            if (g.z_mode == 1) k_z<N, 0><<<grid, TZ, smem_rows<N>(), s>>>(g, md, stage);
            else launch_znl_t<N>(g, md, stage, s);
            break;
        case 1: k_z<N, 1><<<grid, TZ, smem_rows<N>(), s>>>(g, md, stage); break;
        case 3: k_z<N, 3><<<grid, TZ, smem_rows<N>(), s>>>(g, md, stage); break;
        default: k_z<N, 4><<<grid, TZ, smem_rows<N>(), s>>>(g, md, stage); break;
        }
        break;
    }
    case Pass::FX:
        switch (mode) {
        case 0:
            if (g.fx_split == 2) {
                launch_fx_ws_t<N>(g, md, stage, last, s);
            } else if (g.fx_split) {
                k_fwd_x_fft<N, 16><<<dim3(g.NK * g.NZp / 16, 3, g.members), ColCfg<N, 16>::threads,
                                     smem_cols<N, 16>(), s>>>(g);
                k_update<N><<<dim3(update_blocks<N>(), g.members), kUpdThreads, 0, s>>>(g, md, stage, last);
            } else {
                launch_x(pass, mode, g, md, stage, last, arg, s);
            }
            break;
        case 1: k_fwd_x<N, 1, 16><<<grid_state, TC, smem_x<N, 16>(), s>>>(g, md, stage, last); break;
        case 2: k_fwd_x<N, 2, 16><<<grid_state, TC, smem_x<N, 16>(), s>>>(g, md, stage, last); break;
        default: k_fwd_x<N, 3, 16><<<grid_state, TC, smem_x<N, 16>(), s>>>(g, md, stage, last); break;
        }
        break;
    case Pass::ZSTAT: {
        const dim3 grid((unsigned)stats_ctas<N>(), g.members);
        k_z_stats<N><<<grid, 32 * SCfg<N>::WPB, smem_stats<N>(h->nq, h->nt, h->ng), s>>>(g, *h, md);
        break;
    }
    }
}

bool fx_ws() { return has_fx_ws<N>(); }

const SizedOps kOps = {prepare, znl_per_sm, launch, fx_ws};

}  // namespace

template <>
const SizedOps *sized_ops_for<ENS_N>()
{
    return &kOps;
}

}  // namespace ens
