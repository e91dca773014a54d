/*
 * libens: GB300-native ensemble DNS hot path (C ABI).
 *
 * Implements the data-parallel path of the ensemble method of Bentkamp &
 * Wilczek, "Predicting any small-scale statistics of high-Reynolds-number
 * turbulence using ensemble simulations":
 *   - a heterogeneous ensemble of periodic-box Navier-Stokes DNS members that
 *     differ only in their energy injection rate exp(lambda) * eps_bar, with a
 *     forcing that amplifies the velocity Fourier coefficients of a
 *     wavenumber band at every step so that the injection rate is fixed
 *     (Sec. II, Eq. ensemble_hypothesis; Sec. IV);
 *   - per-member velocity-gradient statistics: the joint PDF of
 *     Q = -1/2 Tr A^2 and R = -1/3 Tr A^3 (Sec. V), PDFs of the dissipation
 *     eps = 2 nu Tr S^2 and of the enstrophy omega^2 (Sec. VI), and moments
 *     of the gradient components (Sec. VII, Eq. def_skewness_flatness);
 *   - the mixture over lambda with the Gaussian weights of Sec. IV
 *     (Eq. gaussian_lambda_pdf, one lambda bin per member) or the truncated
 *     Gaussian of the Appendix (Eq. truncated_gaussian).
 *
 * Conventions shared by all calls:
 *   - Box [0, 2 pi)^3, grid x_j = 2 pi j / N.  Forward transform normalised:
 *     uh_k = N^-3 sum_x u(x) exp(-i k.x).
 *   - Host spectral arrays ("full layout") are [3][N][N][N/2+1] complex
 *     doubles (re, im interleaved), index [comp][kx mod N][ky mod N][kz];
 *     modes outside the dealiased set (max_i |k_i| > ceil(N/3) - 1) are zero.
 *   - Host physical arrays are [3][N][N][N] doubles, index [comp][x][y][z].
 *   - The library owns its device memory: either a caller-provided workspace
 *     (size from ens_query; device memory the caller keeps alive until
 *     ens_destroy) or, when workspace is NULL, memory it allocates itself.
 *   - Work is ordered on the CUDA stream given to ens_create.  Calls that
 *     return host data synchronise that stream; the others return at once.
 *   - No exceptions cross the ABI.  Every call returns an ens_status.  A
 *     context remembers its first error ("sticky"); ens_last_error gives the
 *     message.  One context must not be used from two threads at once.
 */
#ifndef ENS_H
#define ENS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ENS_OK = 0,
    ENS_EINVAL = 1,        /* invalid argument (sizes, band, viscosity, ...) */
    ENS_ENOMEM = 2,        /* device memory or workspace too small */
    ENS_ECUDA = 3,         /* a CUDA call failed */
    ENS_ENONFINITE = 4,    /* a member field became non-finite */
    ENS_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    ENS_ESTATE = 6,        /* a member's band energy vanished (forcing undefined) */
    ENS_EUNSUPPORTED = 7   /* grid size without a compiled FFT plan */
} ens_status;

typedef struct ens_ctx ens_ctx;

/* One ensemble member (Sec. IV: same viscosity and forcing band across the
 * ensemble in the paper's setting; the library accepts any per-member
 * values).  N must be one of 16, 32, 64, 128, 256, 384, 512. */
typedef struct {
    int N;               /* grid points per direction */
    int rk_order;        /* 2 or 3: integrating-factor SSP Runge-Kutta order */
    double nu;           /* kinematic viscosity, > 0 */
    double lambda;       /* injection rate exp(lambda) * eps_bar */
    double eps_bar;      /* reference injection rate, > 0 */
    double k_lo, k_hi;   /* forcing band k_lo <= |k| <= k_hi, k_hi <= ceil(N/3)-1 */
    double dt;           /* > 0: fixed time step; <= 0: CFL-adaptive */
    double cfl;          /* CFL number of the adaptive step (Sec. IV: 0.2) */
    double dt_max;       /* cap on the adaptive step, <= 0: none */
    uint64_t seed;       /* seed of the random initial field */
    double init_energy;  /* kinetic energy of the initial field */
} ens_member_desc;

/* Histogram specification (common physical bin edges for all members so
 * that histograms can be mixed).  Q axis in units q0 = eps_norm/(2 nu_norm),
 * R axis in q0^(3/2), tails in log10(eps/eps_norm) and
 * log10(omega^2 nu_norm / eps_norm).  The statistics pass keeps one copy of
 * the counts per CTA in shared memory: ens_create refuses (ENS_EINVAL) a
 * layout that does not fit beside its staged rows (about 180 KB of counts at
 * N = 256, less at N = 128 and 384; 64 x 64 + 2 x 256 bins use 18 KB). */
typedef struct {
    int qr_bins;        /* bins per axis of the Q-R histogram (e.g. 64) */
    double q_lim;       /* Q/q0 in [-q_lim, q_lim) */
    double r_lim;       /* R/q0^1.5 in [-r_lim, r_lim) */
    int tail_bins;      /* bins of each tail histogram (e.g. 256) */
    double tail_lo;     /* log10 axis range [tail_lo, tail_hi) */
    double tail_hi;
    double eps_norm;    /* normalising injection rate */
    double nu_norm;     /* normalising viscosity */
    int grad_bins;      /* bins of each gradient-component histogram, 0..2048 (0: none) */
    double grad_lim;    /* A_ij / sqrt(q0) in [-grad_lim, grad_lim) */
} ens_hist_spec;

/* Per-member counts vector layout (uint64):
 *   [qr_bins*qr_bins | tail_bins (dissipation) | tail_bins (enstrophy) |
 *    8 counters: qr_out, eps_under, eps_over, ens_under, ens_over,
 *                nonfinite, npoints, 0]
 * and, with grad_bins > 0 (gradient-component PDFs, Sec. VI):
 *   [grad_bins (longitudinal A_11, A_22, A_33 pooled) |
 *    grad_bins (transverse A_ij, i != j, pooled) |
 *    4 counters: long_under, long_over, trans_under, trans_over]
 * (3 longitudinal and 6 transverse samples per finite grid point; the
 * mixture divides by 3 n and 6 n.)  ens_counts_len gives the total.
 * Moments (48 doubles per member): sums over points of A_c^p for the nine
 * components c (row-major A_ij = d_j u_i) and p = 2, 3, 4, 6 (index 4c + k),
 * then sums of Q, R, eps, omega^2, Q^2, R^2, eps^2, omega^4, then 4 zeros. */
#define ENS_NMOM 48
#define ENS_NCOUNTERS 8

/* Per-member diagnostics (FP64). */
typedef struct {
    double t;         /* simulated time */
    double dt;        /* last time step */
    double E;         /* kinetic energy 1/2 sum_k |uh_k|^2 */
    double diss;      /* dissipation rate nu sum_k k^2 |uh_k|^2 */
    double EB;        /* energy in the forcing band */
    double P;         /* injected power of the last stage (= exp(lambda) eps_bar) */
    double umax;      /* max_i max_x |u_i| of the last step's first stage */
    double Rlambda;   /* Taylor-scale Reynolds number sqrt(20 E^2 / (3 nu diss)) */
    double kmeta;     /* k_max eta with k_max = N/3, eta = (nu^3/diss)^(1/4) */
    int64_t steps;    /* steps taken */
    int32_t flags;    /* bit 0: non-finite field, bit 1: band energy vanished, bit 2: a device wait gave up */
    int32_t reserved;
} ens_diag;

/* Weight specification of the lambda mixture. */
typedef enum {
    ENS_W_GAUSS_PAPER = 0,  /* Eq. gaussian_lambda_pdf: mean -9cZ/2, variance 9cZ */
    ENS_W_GAUSS = 1,        /* Gaussian with given mean and standard deviation */
    ENS_W_USER = 2,         /* caller-given weights */
    ENS_W_TRUNC_GAUSS = 3   /* Appendix, Eq. truncated_gaussian (c, Z) */
} ens_weight_kind;

typedef struct {
    int kind;              /* ens_weight_kind */
    double c, Z;           /* scaling parameter c and scale gap Z */
    double mu, sigma;      /* ENS_W_GAUSS */
    const double *user;    /* ENS_W_USER: n host weights */
    int renormalize;       /* 1: divide by the covered mass */
} ens_weight_spec;

/* Mixture result; all pointers are caller-owned host buffers (any may be
 * NULL except as noted). */
typedef struct {
    double *weights;     /* [n] member weights (bin masses) */
    double covered;      /* total mass of the members' lambda bins */
    double *pdf_qr;      /* [qr_bins*qr_bins] joint PDF in units of Q/q0, R/q0^1.5 */
    double *pdf_eps;     /* [tail_bins] PDF of log10(eps/eps_norm) */
    double *pdf_ens;     /* [tail_bins] PDF of log10(omega^2 nu_norm/eps_norm) */
    double *moments;     /* [ENS_NMOM] mixed per-point averages */
    double ratios[5];    /* S_long, F_long, F_trans, H_long, H_trans */
    double *pdf_long;    /* [grad_bins] PDF of longitudinal A_ii / sqrt(q0) (may be NULL) */
    double *pdf_trans;   /* [grad_bins] PDF of transverse A_ij / sqrt(q0), i != j (may be NULL) */
} ens_mixture_out;

/* ---- context ---------------------------------------------------------- */

/* Device workspace bytes for ens_create with the same arguments.
 * Errors: ENS_EINVAL / ENS_EUNSUPPORTED on an invalid member. */
ens_status ens_query(const ens_member_desc *members, int n, const ens_hist_spec *hist, size_t *workspace_bytes);

/* Create an ensemble of n members and build each member's seeded random
 * initial field on the device (white noise from splitmix64 + Box-Muller,
 * projected, dealiased, shell spectrum E0(s) ~ s^4 exp(-s^2/2), total
 * energy init_energy).  workspace: device pointer of at least
 * ens_query() bytes, or NULL for library-owned memory.  stream: a
 * cudaStream_t (NULL: legacy default stream).  On failure *out is NULL. */
ens_status ens_create(const ens_member_desc *members, int n, const ens_hist_spec *hist, void *workspace,
                      size_t workspace_bytes, void *stream, ens_ctx **out);
ens_status ens_destroy(ens_ctx *ctx);
const char *ens_last_error(const ens_ctx *ctx);
const char *ens_status_string(ens_status s);

/* ---- time stepping (Sec. IV) -------------------------------------------- */

/* Advance every member by nsteps steps (asynchronous on the context stream;
 * one CUDA-graph replay per step).  Each step: one RK stage after another,
 * each stage = inverse transforms of u and omega = i k x u, the rotational
 * nonlinear term u x omega with 2/3 dealiasing and max|u| for the CFL step,
 * forward transforms, Leray projection, constant-power band forcing
 * alpha u with alpha = exp(lambda) eps_bar / (2 E_B), and the
 * integrating-factor SSP-RK stage update. */
ens_status ens_step(ens_ctx *ctx, int nsteps);
/* Same, launching the kernels directly instead of replaying a graph. */
ens_status ens_step_nograph(ens_ctx *ctx, int nsteps);
/* Same results, launched the slow way for comparison: one member at a time,
 * every pass of every member a separate launch on the context stream. */
ens_status ens_step_sequential(ens_ctx *ctx, int nsteps);
/* One step (the step of ens_step, Sec. IV) of an ensemble whose state lives
 * in host memory: host_in holds the state in the layout of ens_get_state
 * (bytes >= ens_state_bytes), the stepped state is written to host_out
 * (host_out may equal host_in).  The members go through in chunks of
 * `chunk` members of one grid size (0: per group, sizes growing by a factor
 * 3 from one member up to a third of the group, the middle in chunks of at
 * most that and the same sizes shrinking at the end, e.g. 1 3 9 19 19 9 3 1
 * for 64 members, so that the pipeline fills and drains quickly): a
 * chunk's upload,
 * its energy sums (as after ens_set_state), its
 * three RK stages and its download are ordered on the device, and the
 * upload of the next chunk and the download of the previous one run on two
 * copy streams while a chunk computes.  Overlap needs page-locked host
 * memory; pageable memory gives the same results without it.  The device
 * copy of the state and the diagnostics end as after ens_set_state,
 * ens_step and ens_get_state, to FP32 rounding (bit for bit where each
 * member's z-pass rows go through the same warp streams in a chunk as in
 * the whole group: the z pass pairs the n_z rows of a stream into one
 * complex line); the call returns once host_out is written.
 * ENS_EINVAL for null buffers, too few bytes or chunk < 0. */
ens_status ens_step_host(ens_ctx *ctx, const void *host_in, void *host_out, size_t bytes, int chunk);

/* ---- autotuning (no counterpart in the paper: launch shapes of this
 * library's kernels) ------------------------------------------------------ */

/* Per grid-size group: the variants of the stage passes.
 *   tile_x, tile_y  columns per CTA of the x / y FFT passes (8 or 16);
 *   plan_x          FFT plan of the x passes: 0 the default radix plan,
 *                   1 (N = 128, 256, 512 only) a plan with twice the
 *                   threads per line and a tighter register budget
 *                   (128: 8x2x8, 256: 8x4x8, 512: 8x8x8 on 64 threads);
 *   fx_split        0: the last pass of a stage fused (forward x transform,
 *                   projection, forcing, RK update in one launch); 1: two
 *                   launches (transform into a compact spectral buffer, then
 *                   a streaming update), more HBM bytes, lighter kernels;
 *                   2 (N = 256 only): fused, in persistent CTAs of two warp
 *                   groups (one transforms a column tile while the other
 *                   updates the previous tile, its state reads overlapping
 *                   the transforms; the fields and sums of fx_split 0 with
 *                   16-column tiles, bit for bit);
 *   z_variant       0: persistent TMA-pipelined z pass with z_ctas_per_sm
 *                   CTAs per SM (1 .. the kernel's occupancy limit),
 *                   1: one CTA per group of rows (z_ctas_per_sm unused
 *                   but kept, and checked, for a switch back to 0),
 *                   2 (N = 256 only): the persistent pass with a two-pass
 *                   16 x 16 warp plan (one shared-memory exchange per line
 *                   instead of two; z_ctas_per_sm up to its own limit).
 * Every variant computes the same transforms; the FP64 energy sums of the
 * update pass are accumulated over tile_x-dependent CTA partials, so
 * changing tile_x changes their rounding order (fields agree to FP32
 * rounding, not bit for bit). */
#define ENS_MAX_GROUPS 8
typedef struct {
    int N;               /* grid size (read-only: must match the context) */
    int tile_x, tile_y;
    int z_variant;
    int z_ctas_per_sm;
    int plan_x;
    int fx_split;
} ens_group_tuning;
typedef struct {
    int groups;          /* number of grid-size groups (read-only) */
    int parallel_groups; /* 1: groups as parallel graph branches; 0: one chain */
    int persistent;      /* 1: every member of every grid size advances one RK
                          * stage in one persistent launch (a cooperative grid of
                          * one CTA per SM taking work items -- column tiles,
                          * z-pass row-group chunks, stage finishes -- in
                          * dependency order, waiting, bounded, on per-member
                          * pass counters); available when every grid size is
                          * 128, 256 or 384; the group variants below are then
                          * ignored (16-column tiles, 16 threads per FFT line,
                          * the default z warp plan, the fused last pass) */
    ens_group_tuning group[ENS_MAX_GROUPS];   /* ascending N */
    double ms_per_step;  /* ens_autotune: mean step time of the winner, else 0 */
    int trials;          /* ens_autotune: configurations timed */
} ens_tuning;
/* Current tuning (defaults at creation: tiles 16, persistent z pass at its
 * occupancy limit, parallel groups). */
ens_status ens_get_tuning(const ens_ctx *ctx, ens_tuning *out);
/* Install a tuning (for instance one cached from an earlier ens_autotune on
 * the same device and member set).  ENS_EINVAL (not sticky, previous tuning
 * kept) if a field is out of range or the groups do not match.  Synchronises;
 * the next ens_step captures a new graph. */
ens_status ens_set_tuning(ens_ctx *ctx, const ens_tuning *t);
/* Time the variants on this context's own members and install the fastest:
 * coordinate descent in two sweeps, each over parallel_groups and then, for
 * each group, plan_x, tile_x, tile_y, the z variant and its CTAs per SM and
 * fx_split (0, 1, 2); then persistent
 * (where available); each trial restores the member
 * state from a device snapshot, runs one untimed step and times `steps`
 * graph replays with CUDA events; a candidate wins only if it is more than
 * 1% faster.  The member state is restored afterwards (the simulation does
 * not advance).  Needs device memory for one copy of the spectral state
 * (ENS_ENOMEM otherwise, context unchanged).  out (may be NULL) receives
 * the installed tuning with ms_per_step and trials. */
ens_status ens_autotune(ens_ctx *ctx, int steps, ens_tuning *out);

/* ---- statistics (Secs. V-VII) ---------------------------------------- */

/* One snapshot of every member: gradient fields, invariants, histograms and
 * moments.  accumulate = 0 clears the member statistics first. */
ens_status ens_gradient_stats(ens_ctx *ctx, int accumulate);
/* Copy statistics to the host: counts [n][counts_len] (uint64), moments
 * [n][ENS_NMOM]; either may be NULL.  Synchronises. */
ens_status ens_get_stats(ens_ctx *ctx, uint64_t *counts, double *moments);
/* counts_len of a histogram specification. */
int ens_counts_len(const ens_hist_spec *hist);
/* The statistics pass's bin rule alone (a check of the rule, used by the
 * tests): values[0..n) already in an axis's units -- axis 0 Q/q0, 1
 * R/q0^(3/2), 2 the log10 tail axis (eps/eps_norm, omega^2 nu_norm/eps_norm),
 * 3 A_ij/sqrt(q0) (needs grad_bins > 0) -- binned on the device with the
 * context's FP32 edges by the same device code as ens_gradient_stats: bins[i]
 * = b iff edge[b] <= values[i] < edge[b+1], -1 below the first edge (and a
 * non-positive value on the log axis), the axis's bin count at or above the
 * last.  Host buffers, caller-owned; synchronous.  ENS_EINVAL for another
 * axis, n < 0 or a null buffer with n > 0. */
ens_status ens_bin_check(ens_ctx *ctx, int axis, const float *values, int n, int *bins);

/* ---- mixture (Sec. II, Eq. pdf_superposition; Sec. IV) ---------------- */

/* Mix the context's current member statistics with lambda weights.
 * Synchronises.  Errors: ENS_EINVAL on a bad weight spec. */
ens_status ens_mixture(ens_ctx *ctx, const ens_weight_spec *w, ens_mixture_out *out);
/* Mix statistics gathered elsewhere (e.g. from several processes): host
 * inputs lambdas [n], counts [n][counts_len], moments [n][ENS_NMOM]; runs on
 * the device with temporary device memory on `stream`.  n <= 1024. */
ens_status ens_mixture_host(int n, const double *lambdas, const uint64_t *counts, const double *moments,
                            const ens_hist_spec *hist, const ens_weight_spec *w, ens_mixture_out *out,
                            void *stream);

/* Same mixture as ens_mixture_host, for callers that cannot allocate device
 * memory: for instance a process whose GPU memory is entirely reserved by
 * another allocator (a framework's caching allocator that has claimed the
 * device), or an application that budgets every device byte up front.  The
 * paper has no counterpart; this is a deployment convenience.
 *
 * It allocates nothing (no cudaMalloc, cudaMallocAsync or cudaFree, no
 * allocating library call): inputs and results pass through one fixed
 * scratch array compiled into the library, of about 4.3 MB, which every GPU
 * that loads the library holds until the process exits.  Limits:
 * n <= ENS_NOALLOC_MAX_MEMBERS and ens_counts_len(hist) <=
 * ENS_NOALLOC_MAX_COUNTS; larger requests return ENS_EINVAL with a message
 * on stderr (use ens_mixture_host for them).
 *
 * The first call on a device, made while that device is current, looks up
 * the scratch array's device address (cudaGetSymbolAddress).  All calls on a
 * device share the one array and it keeps the last call's contents: calls
 * that overlap on the GPU (from several threads or streams at once) race and
 * give wrong results.  The call synchronises `stream` before it returns, so calls made
 * one after another from one thread do not overlap. */
#define ENS_NOALLOC_MAX_MEMBERS 64
#define ENS_NOALLOC_MAX_COUNTS 8192
ens_status ens_mixture_host_noalloc(int n, const double *lambdas, const uint64_t *counts, const double *moments,
                                    const ens_hist_spec *hist, const ens_weight_spec *w, ens_mixture_out *out,
                                    void *stream);

/* ---- scaling-exponent theory (Secs. III, V, VII) ----------------------- */

/* Inertial-range exponent families zeta_p:
 *   ENS_ZETA_QUADRATIC  zeta_p = p/3 - c (p^2 - 3p)/2 (Sec. IV, Eq.
 *                       quadratic_scaling_exponents; Gaussian lambda); c >= 0
 *   ENS_ZETA_LOGPOISSON zeta_p = p/9 + C0 (1 - beta^(p/3)) (a literature
 *                       parameterization of the kind listed in Sec. III;
 *                       beta = 2/3, C0 = 2 give zeta_3 = 1); 0 < beta < 1,
 *                       C0 > 0
 *   ENS_ZETA_RATIONAL   zeta_p = (1 + 3 beta) p / (3 (1 + beta p)) (Yakhot's
 *                       saturating mean-field form, beta ~ 0.05; the kind of
 *                       saturating exponents Sec. VII inverts numerically);
 *                       beta > 0
 * The cumulant generating function of lambda is K(t; Z) = (t - zeta_3t) Z
 * (Sec. III, Eq. exponents_KZ_1). */
typedef enum { ENS_ZETA_QUADRATIC = 0, ENS_ZETA_LOGPOISSON = 1, ENS_ZETA_RATIONAL = 2 } ens_zeta_kind;
typedef struct {
    int kind;
    double c;     /* quadratic */
    double beta;  /* log-Poisson and rational */
    double C0;    /* log-Poisson */
} ens_zeta_spec;

/* Uniform lambda grid of the numerical inversion: ENS_LAMBDA_GRID points
 * lambda_j = LO + j (HI - LO) / ENS_LAMBDA_GRID, j = 0 .. GRID-1. */
#define ENS_LAMBDA_GRID 65536
#define ENS_LAMBDA_GRID_LO (-30.0)
#define ENS_LAMBDA_GRID_HI 30.0

/* P(lambda; Z) on the grid above (host array of ENS_LAMBDA_GRID doubles) by
 * the numerical inverse two-sided Laplace transform of exp K (Sec. VII):
 * exp K(i s) sampled at the grid's conjugate frequencies, then an FP64 FFT
 * on the device.  Saturating exponents (zeta_p -> zeta_inf) give P a point
 * mass exp(-zeta_inf Z) at lambda_max = Z (Appendix, saturation): it is
 * removed from exp K before the transform, and the returned P is the
 * continuous part.  Quadratic and rational families (log-Poisson lambda is
 * a lattice: ENS_EINVAL).  Z > 0.  Synchronises `stream` (NULL: legacy
 * default stream). */
ens_status ens_lambda_pdf(const ens_zeta_spec *zeta, double Z, double *pdf, void *stream);
/* Member weights w_i (host arrays of n doubles) for the lambda distribution
 * of `zeta` at scale gap Z > 0: the mass of P(lambda; Z) in each member's
 * lambda bin (bin edges halfway between neighbouring distinct lambdas, the
 * outer bins as wide as their inner half; a shared lambda value splits its
 * bin's mass equally).  Quadratic and rational families: trapezoid
 * integral of ens_lambda_pdf over the bin, bin ends interpolated linearly,
 * clipped to the grid, plus the point mass at lambda = Z of the rational
 * family in the bin that holds it (lo <= Z < hi).  Log-Poisson: exact, lambda = 2Z/3 + k ln(beta) with
 * k ~ Poisson(C0 Z), k < 400.  Not renormalised; *covered (may be NULL) is
 * their sum.  Pass the result to ens_mixture as ENS_W_USER weights.
 * Synchronises `stream`.  ENS_EINVAL for non-finite inputs or parameters
 * outside the family's range. */
ens_status ens_lambda_weights(const ens_zeta_spec *zeta, double Z, int n, const double *lambdas, double *weights,
                              double *covered, void *stream);
/* Gradient-moment exponents rho_m = m - zeta_{m + rho_m} (Sec. III, Eq.
 * nelkin_rhom) for nm orders m; FP64 bisection (host). */
ens_status ens_nelkin_exponents(const ens_zeta_spec *zeta, int nm, const double *m, double *rho);
/* Predicted R_lambda exponents of skewness, flatness and hyper-flatness of
 * the gradient components (Sec. VII): 2rho3 - 3rho2, 2rho4 - 4rho2,
 * 2rho6 - 6rho2; out holds 3 doubles. */
ens_status ens_ratio_exponents(const ens_zeta_spec *zeta, double *out);
/* Scale gap for a target R_lambda (Sec. V): fit ln R_lambda = ln R0 +
 * lambda/6 over the members with lambda >= 0 (constant C_eps, Eq.
 * Re_definition), then Z = 1.5 ln(R_ref / R0) (Eq. Rlambda_Z_relation).
 * Host arithmetic; R0 may be NULL. */
ens_status ens_scale_gap(int n, const double *lambdas, const double *rlambda, double R_ref, double *Z, double *R0);

/* Change a member's time-step rule from the next step on (dt > 0: fixed dt;
 * otherwise CFL with number cfl > 0, capped at dt_max if dt_max > 0), for
 * instance to retry a member that went non-finite with a smaller CFL number.
 * The member's description (and so checkpoint compatibility) is unchanged;
 * the rule itself is part of the run state that ens_save writes.
 * Synchronises. */
ens_status ens_set_timestep(ens_ctx *ctx, int member, double dt, double cfl, double dt_max);

/* ---- checkpoint / resume ------------------------------------------------ */

/* Write the whole ensemble to a file: member descriptions, the spectral
 * state (FP32 compact layout), every member's run state (time, step count,
 * dt, energy sums, forcing amplitude, CFL maxima, flags), the accumulated
 * histogram counts and moment sums, and an FNV-1a checksum of all of it.
 * Written to path.tmp and renamed, so an interrupted save leaves no partial
 * file under path.  The format is this library's (host byte order; not an
 * interchange format).  Synchronises. */
ens_status ens_save(ens_ctx *ctx, const char *path);
/* Resume from ens_save's file into a context created with the same members
 * (every ens_member_desc field equal), histogram specification and RK
 * order: continuing from the loaded state gives the same fields, bit for
 * bit, as continuing the saved context (under the same tuning).  ENS_EINVAL
 * (not sticky; context unchanged) for a missing, foreign, truncated or
 * corrupted file, with the reason in ens_last_error.  Synchronises. */
ens_status ens_load(ens_ctx *ctx, const char *path);

/* ---- state access ------------------------------------------------------ */

/* Member spectral field <-> host full layout (FP64; converted from/to the
 * library's FP32 compact layout).  Synchronises.  Uploading recomputes the
 * member's spectral sums and forcing amplitude. */
ens_status ens_get_field(ens_ctx *ctx, int member, double *host_spec);
ens_status ens_set_field(ens_ctx *ctx, int member, const double *host_spec);
/* The whole ensemble state in the library's FP32 compact layout, as raw
 * bytes (ens_state_bytes of them), to/from host memory (pinned memory
 * recommended).  Synchronises. */
size_t ens_state_bytes(const ens_ctx *ctx);
ens_status ens_get_state(ens_ctx *ctx, void *host, size_t bytes);
ens_status ens_set_state(ens_ctx *ctx, const void *host, size_t bytes);
/* Physical velocity of a member (inverse transforms on the device) /
 * spectral field from a physical velocity (forward transforms on the
 * device, dealiased; no projection).  Host physical layout.  Synchronise. */
ens_status ens_get_velocity(ens_ctx *ctx, int member, double *host_phys);
ens_status ens_set_velocity(ens_ctx *ctx, int member, const double *host_phys);
/* Right-hand side F(u) = P N(u) + alpha u 1_B of every member at its
 * current state, returned for one member in the host full layout. */
ens_status ens_rhs(ens_ctx *ctx, int member, double *host_spec);

/* Diagnostics of every member (n entries).  Synchronises.  Returns
 * ENS_ETIMEOUT, ENS_ENONFINITE or ENS_ESTATE, in that order of precedence,
 * if a member is flagged (the array is still filled); flags bit 2 marks a
 * member whose rows a device-side wait gave up on (ENS_ETIMEOUT; its state
 * is then invalid). */
ens_status ens_diagnostics(ens_ctx *ctx, ens_diag *out);
ens_status ens_synchronize(ens_ctx *ctx);

/* Failure-detection test hook (no counterpart in the paper).  Arms the next
 * ens_step_nograph call (one-shot): in its persistent z passes the bulk
 * copies of `member`'s first row group are not issued, and the wait on that
 * group's barrier gives up after wait_polls polls (1 .. 65536) instead of
 * the full limit, so the bounded wait runs out with nothing in flight; every
 * other wait, on copies that were issued, keeps its full limit.  The warp
 * that gives up leaves its remaining rows unprocessed and flags `member` and
 * every later member of its grid-size group (flags bit 2); ens_diagnostics
 * then returns ENS_ETIMEOUT.  The context stays usable (the flagged states
 * are invalid).  ENS_EINVAL (not sticky) for a member out of range, a
 * wait_polls out of range, or a member whose group runs the z pass variant
 * without bulk copies (z_variant 1). */
ens_status ens_test_skip_copy(ens_ctx *ctx, int member, int wait_polls);

/* ---- learned lambda interpolant (surrogate) ------------------------------
 * A 4-layer MLP (width 256, SiLU; BF16 weights, FP32 accumulation on the
 * tcgen05 tensor cores, FP32 master weights, Adam) that maps (bin, lambda) to
 * a logit; a softmax over the bins of each PDF kind gives the per-lambda
 * densities of the joint Q-R histogram and of the two tail histograms.  It
 * lets the lambda mixture of Sec. II (Eq. ensemble_hypothesis) and Sec. IV
 * (Eq. gaussian_lambda_pdf) be evaluated on a fine lambda quadrature between
 * the simulated members; the member quadrature (ens_mixture) remains the
 * reference and measures its error.  The paper itself mixes member statistics
 * directly; the interpolant is this library's addition.
 *
 * Row features of (bin, lambda): bin centre coordinates scaled to [-1, 1]
 * (Q and R for the joint PDF, the log axis for the tails), lambda / 5, a
 * one-hot PDF kind, and sin/cos(pi k s) of the three coordinates for
 * k = 1..4 (31 features, padded to 64).  Targets: each member's in-range
 * histogram of each kind normalised to unit sum; loss: mean over (member,
 * kind) of the cross-entropy -sum_b p_b log q_b.  Parameters (FP32, this
 * order): W1 [256][64], b1 [256], W2 [256][256], b2, W3 [256][256], b3,
 * w4 [256], b4 [1].  Work runs on `stream`; calls returning host data
 * synchronise it.  Device memory is allocated by the object. */
typedef struct ens_surrogate ens_surrogate;
ens_status ens_surrogate_create(uint64_t seed, void *stream, ens_surrogate **out);
ens_status ens_surrogate_destroy(ens_surrogate *s);
size_t ens_surrogate_param_count(void);
ens_status ens_surrogate_get_params(ens_surrogate *s, float *host);
ens_status ens_surrogate_set_params(ens_surrogate *s, const float *host);
/* Loss and gradient (FP32, parameter order above) of the current parameters
 * on n members' histograms (counts layout of ens_get_stats). */
ens_status ens_surrogate_loss_grad(ens_surrogate *s, int n, const double *lambdas, const uint64_t *counts,
                                   const ens_hist_spec *hist, double *loss, float *grad);
/* `steps` full-batch Adam steps on the members' histograms, the learning
 * rate decaying along a cosine from lr at the first step of the call to
 * lr / 20 at its last; *final_loss is the loss of the last step's forward
 * pass. */
ens_status ens_surrogate_train(ens_surrogate *s, int n, const double *lambdas, const uint64_t *counts,
                               const ens_hist_spec *hist, int steps, double lr, double *final_loss);
/* Densities (bin probabilities) at n lambda values: probs [n][qr_bins^2 +
 * 2 tail_bins], each kind summing to one.  Inference (here and in
 * ens_surrogate_mixture) runs the fused kernel: per 128-row tile the
 * features, the three tcgen05 layers with bias + SiLU epilogues from TMEM and
 * the head, activations kept in shared memory, weights streamed in by bulk
 * copies. */
ens_status ens_surrogate_density(ens_surrogate *s, int n, const double *lambdas, const ens_hist_spec *hist,
                                 double *probs);
/* Mixture over a midpoint lambda quadrature of nquad points on
 * [lam_lo, lam_hi] with the masses of a Gaussian weight specification
 * (ENS_W_GAUSS_PAPER or ENS_W_GAUSS), renormalised; fills pdf_qr, pdf_eps,
 * pdf_ens of `out` (same units as ens_mixture). */
ens_status ens_surrogate_mixture(ens_surrogate *s, const ens_hist_spec *hist, const ens_weight_spec *w,
                                 double lam_lo, double lam_hi, int nquad, ens_mixture_out *out);
/* Average device time (ms, CUDA events on the object's stream) of one
 * hidden-layer GEMM of `rows` rows (rows x 256 x 256, BF16 in, FP32 out). */
ens_status ens_surrogate_time_gemm(ens_surrogate *s, long long rows, int iters, double *ms);
/* Logits [n][qr_bins^2 + 2 tail_bins] at n lambda values from the fused
 * inference kernel (fused != 0) or the layer-by-layer forward pass that
 * training uses (fused == 0); both round activations to BF16 the same way. */
ens_status ens_surrogate_logits(ens_surrogate *s, int n, const double *lambdas, const ens_hist_spec *hist, int fused,
                                float *logits);
/* Average device time (ms) of one fused inference launch over nquad lambda
 * values of this histogram layout (nquad (qr_bins^2 + 2 tail_bins) rows;
 * 2 (64 + 2 x 256 + 1) 256 flops per row). */
ens_status ens_surrogate_time_infer(ens_surrogate *s, const ens_hist_spec *hist, int nquad, int iters, double *ms);
/* Tensor-core GEMM check C = A B^T on host BF16 bit patterns: A [M][K],
 * B [N][K], C [M][N] FP32; M % 128 == 0, N % 64 == 0, K % (64 ksplit) == 0,
 * ksplit <= 32 splits K across CTAs (partials summed in a fixed order). */
ens_status ens_tc_gemm_check(const uint16_t *A, const uint16_t *B, float *C, int M, int N, int K, int ksplit);

/* ---- introspection / profiling ----------------------------------------- */

/* Number of members, grid size of a member. */
int ens_members(const ens_ctx *ctx);
int ens_member_n(const ens_ctx *ctx, int member);
/* Launch one pass of one RK stage for every member (profiling): pass 0 IX,
 * 1 IY, 2 ZNL, 3 FY, 4 FXU.  Asynchronous. */
ens_status ens_run_pass(ens_ctx *ctx, int pass, int stage);
/* Kernels one ens_step launches per step (graph nodes; with the persistent
 * stage kernel, one per RK stage). */
int ens_kernels_per_step(const ens_ctx *ctx);
/* Algorithmic HBM bytes of one pass for all members (unique bytes read +
 * written, valid modes only); pass as in ens_run_pass, stage 0..2; pass 5
 * is one ens_gradient_stats snapshot (stage ignored). */
double ens_pass_bytes(const ens_ctx *ctx, int pass, int stage);

#ifdef __cplusplus
}
#endif
#endif
