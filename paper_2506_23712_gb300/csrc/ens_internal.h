// Internal types shared by the kernels and the C-ABI layer of libens.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ens {

constexpr int kTile = 16;        // column padding of the layouts; widest column tile of the strided-axis passes
constexpr int kFields = 8;       // fields per member in the pass buffers
constexpr int kNMom = 48;        // gradient moment sums per member
constexpr int kUpdChunk = 2048;  // modes per CTA of the split update pass (256 threads x 8)

// Per-member parameters and run state, resident in device memory.
struct MemberDev {
    // parameters (Sec. IV: same band and viscosity, injection exp(lambda) eps_bar)
    double nu, eps_inj, klo2, khi2;
    double dt_fixed, cfl, dt_max;
    int rk, N;
    int group, index_in_group;
    unsigned long long seed;     // initial-field seed
    double init_energy;
    int nblk;                    // CTAs writing FP64 partial sums for this member
    int band_lo2, band_hi2;      // forcing band as integer bounds on |k|^2
    int pad0;
    // run state
    double t, dt, E, diss, EB, alpha, P, umax;
    long long steps;
    unsigned int umax_bits[4];   // max |u_i| per RK stage, as float bits
    int flags;                   // bit 0: non-finite field, bit 1: band energy vanished
    int pad;
};

enum : int { kFlagNonFinite = 1, kFlagNoBandEnergy = 2, kFlagTimeout = 4 };

// Geometry of one group of members sharing a grid size N.
//   state  U, S : [member][3][NK][NK][NZp]     (kx, ky, kz; compact dealiased)
//   buffer A    : [member][kFields][NK][N][NZp] (ky, x, kz)
//   buffer B    : [member][kFields][N][N][NZp]  (y, x, kz)
struct Geo {
    int N, kc, NK, NZ, NZp;
    int members;       // members in the group
    int first;         // global index of the group's first member
    long long sU;      // complex values per state component: NK*NK*NZp
    long long sA;      // per buffer-A field: NK*N*NZp
    long long sB;      // per buffer-B field: N*N*NZp
    float2 *U, *S, *A, *B;
    const float2 *tw;  // W_N^m = exp(-2 pi i m / N), m < N
    double *partial;   // per-CTA FP64 partial sums [member][blocks][4]
    int partial_blocks;
    double *shell;     // initial-field shell sums [member][shells]
    int shells;
    unsigned long long *counts;  // statistics counts [member][counts_len]
    double *mom_partial;         // per-CTA moment partials [member][blocks][kNMom]
    int mom_blocks;
    // tuning of the stage passes (chosen by the autotuner)
    int tile_x, tile_y;          // columns per CTA of the x / y passes (8 or 16)
    int plan_x;                  // FFT plan of the x passes (0: default, 1: more threads per line)
    int fx_split;                // last pass of a stage: 0 fused, 1 transform + update launches,
                                 // 2 fused with the two halves in overlapping warp groups
    int z_mode;                  // 0: persistent TMA z pass, 1: one CTA per row group
    int z_ctas;                  // persistent CTAs of the z-direction nonlinear pass
    int sms;                     // streaming multiprocessors of the device (persistent launches)
    // failure test only (ens_test_skip_copy): the persistent z pass issues no
    // bulk copy for the first row group of this member (local index in the
    // group; -1: none) and waits for that group's barrier at most
    // z_skip_wait polls, so the bounded wait gives up; every other wait keeps
    // its full limit
    int z_skip_member;
    int z_skip_wait;
};

struct HistDev {
    int nq, nt, counts_len;
    float q_scale, r_scale;      // 1/q0, 1/q0^1.5
    float eps_scale, ens_scale;  // 1/eps_norm, nu_norm/eps_norm
    float q_lo, q_inv_w, r_lo, r_inv_w;
    float t_lo, t_inv_w;         // log10 axis
    const float *edges_q, *edges_r, *edges_t;  // FP32 edges (nq+1, nq+1, nt+1)
    int ng;                      // gradient-component bins (0: none)
    float g_scale, g_lo, g_inv_w;  // 1/sqrt(q0); linear axis
    const float *edges_g;        // FP32 edges (ng+1)
};

// [nq*nq | nt | nt | 8 counters] then, with ng > 0, [ng | ng | 4 counters]
inline long long counts_len_of(int nq, int nt, int ng)
{
    return (long long)nq * nq + 2LL * nt + 8 + (ng > 0 ? 2LL * ng + 4 : 0);
}

}  // namespace ens
