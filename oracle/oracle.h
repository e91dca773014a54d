/*
 * FP64 CPU oracle for the ensemble DNS hot path (Bentkamp & Wilczek,
 * "Predicting any small-scale statistics of high-Reynolds-number turbulence
 * using ensemble simulations").
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library
 * against a plain, slow, obviously correct restatement of the method.  Only
 * the test suite, the smoke entry point and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * Conventions (Sec. IV; readings where the paper is silent are marked [R]):
 *   - box [0, 2pi)^3, grid x_j = 2 pi j / N, integer wavenumbers;
 *   - [R] forward transform normalised: uh_k = N^-3 sum_x u(x) exp(-i k.x),
 *     so that E = 1/2 <|u|^2> = 1/2 sum_k |uh_k|^2 over the full spectrum;
 *   - spectral arrays use the standard real-to-complex layout
 *     [x][y][kz] with kz in [0, N/2], complex doubles interleaved (re, im);
 *   - physical arrays are [x][y][z] doubles;
 *   - a field with several components stores them one after the other.
 */
#ifndef ENS_ORACLE_H
#define ENS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- FFT (own mixed-radix Cooley-Tukey, FP64) -------------------------- */
/* In-place complex DFT of length n (any n; radix 2/3 recursion, direct DFT
 * for other prime factors).  sign = -1: exp(-i...), sign = +1: exp(+i...).
 * Unnormalised. data: 2n doubles (re, im). */
void or_fft1(double *data, int n, int sign);
/* Forward 3D real-to-complex transform, normalised by N^-3.
 * u: N^3 doubles; uh: N*N*(N/2+1) complex. */
void or_rfft3(const double *u, double *uh, int N);
/* Inverse 3D complex-to-real transform (unnormalised synthesis
 * u(x) = sum_k uh_k exp(i k.x)); the kz = 0 and kz = N/2 planes enter
 * through their real parts only (Hermitian extension). */
void or_irfft3(const double *uh, double *u, int N);

/* ---- member description ------------------------------------------------ */
typedef struct {
    int N;              /* grid points per direction (factors 2 and 3 only) */
    int rk_order;       /* 2 or 3 */
    double nu;          /* kinematic viscosity */
    double lambda;      /* log injection factor: eps_inj = exp(lambda)*eps_bar */
    double eps_bar;     /* reference injection rate */
    double k_lo, k_hi;  /* forcing band, |k| in [k_lo, k_hi] (inclusive) */
    double dt;          /* > 0: fixed step; <= 0: CFL-adaptive */
    double cfl;         /* CFL number for the adaptive step */
    double dt_max;      /* cap on the adaptive step (<= 0: no cap) */
    uint64_t seed;      /* initial-field seed */
    double init_energy; /* initial kinetic energy */
} or_member;

typedef struct {
    double t;       /* time after the step(s) */
    double dt;      /* last step size */
    double E;       /* kinetic energy 1/2 sum |uh|^2 */
    double diss;    /* dissipation nu sum k^2 |uh|^2 */
    double EB;      /* band energy 1/2 sum_{k in B} |uh|^2 */
    double P;       /* injected power of the last stage evaluated */
    double umax;    /* max_i max_x |u_i| of the last step's initial field */
} or_diag;

/* Largest kept wavenumber of the cubic 2/3 rule: ceil(N/3) - 1. */
int or_kc(int N);
/* Number of full-spectrum modes in the forcing band (Hermitian pairs
 * counted twice). */
int or_band_modes(int N, double k_lo, double k_hi);

/* Seeded random initial field (3 components, spectral layout). */
void or_initial_field(const or_member *m, double *uh);
/* Counter-based white noise used by the initial field: value of component c
 * at flat index idx, from splitmix64 + Box-Muller (FP64). */
double or_white_noise(uint64_t seed, uint64_t counter);

/* Right-hand side F(uh) = P N(uh) + f(uh) of the spectral equation
 * (3 components).  Optional outputs (may be NULL): nl = projected,
 * dealiased nonlinear term alone; umax; alpha (forcing amplitude). */
void or_rhs(const or_member *m, const double *uh, double *F, double *nl,
            double *umax, double *alpha);
/* Spectral sums of a state: E, dissipation, band energy. */
void or_sums(const or_member *m, const double *uh, double *E, double *diss,
             double *EB);
/* Advance nsteps steps (IF-RK2 or IF-RK3).  *t is advanced.  Returns 0, or
 * -1 if the band energy vanished, -2 on a non-finite field. */
int or_step(const or_member *m, double *uh, int nsteps, double *t, or_diag *d);

/* ---- gradient statistics ----------------------------------------------- */
typedef struct {
    int qr_bins;      /* bins per axis of the joint Q-R histogram */
    double q_lim;     /* Q / q0 in [-q_lim, q_lim) */
    double r_lim;     /* R / q0^(3/2) in [-r_lim, r_lim) */
    int tail_bins;    /* bins of the dissipation / enstrophy histograms */
    double tail_lo;   /* log10 range [tail_lo, tail_hi) */
    double tail_hi;
    double eps_norm;  /* eps_bar of the normalisation */
    double nu_norm;   /* nu of the normalisation */
    int grad_bins;    /* bins of each gradient-component histogram (0: none) */
    double grad_lim;  /* A_ij / sqrt(q0) in [-grad_lim, grad_lim) */
} or_hist_spec;

/* Counts layout: [qr_bins^2 | tail_bins (dissipation) | tail_bins
 * (enstrophy) | 8 counters], counters = {qr_out, eps_under, eps_over,
 * ens_under, ens_over, nonfinite, npoints, 0}; with grad_bins > 0 followed
 * by [grad_bins (longitudinal A_11, A_22, A_33 pooled) | grad_bins
 * (transverse A_ij, i != j, pooled) | 4 counters: long_under, long_over,
 * trans_under, trans_over]. */
int or_counts_len(const or_hist_spec *h);
/* the histogram bin rule on values in an axis's units (axis 0 Q, 1 R,
 * 2 log10 tail, 3 gradient component): -1 underflow, n overflow */
void or_bin_values(const or_hist_spec *h, int axis, const float *x, long n, int *out);
#define OR_NMOM 48
/* Velocity-gradient fields A_ij = d_j u_i (9 physical fields, row-major ij). */
void or_gradient(const double *uh, int N, double *A);
/* Per-point invariants from the 9 gradient fields: Q, R, eps, omega^2
 * (each N^3; any output may be NULL). */
void or_invariants(const double *A, int N, double nu, double *Q, double *R,
                   double *eps, double *ens);
/* Accumulate histograms and moments of one snapshot. */
void or_gradient_stats(const double *uh, int N, double nu,
                       const or_hist_spec *h, uint64_t *counts,
                       double *moments);

#ifdef __cplusplus
}
#endif
#endif
