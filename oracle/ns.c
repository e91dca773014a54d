/*
 * Oracle Navier-Stokes member solver, FP64.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * One ensemble member is forced, statistically stationary turbulence in a
 * periodic box whose energy injection rate is fixed to exp(lambda)*eps_bar by
 * a forcing that amplifies the Fourier coefficients of a wavenumber band at
 * every step (Sec. II, Eq. ensemble_hypothesis; Sec. IV).  The paper names no further
 * numerics; the readings used here ([R]) are:
 *   - rotational form: d_t u = u x omega - grad(p + |u|^2/2) + nu lap u + f,
 *     div u = 0, i.e. d_t uh = P(k) FFT[u x omega] + fh - nu k^2 uh with the
 *     Leray projector P_ij = delta_ij - k_i k_j / k^2 and uh(0) = 0;
 *   - cubic 2/3 dealiasing: keep a mode iff max_i |k_i| <= ceil(N/3) - 1;
 *   - forcing fh = alpha uh on B = {k_lo <= |k| <= k_hi}, with
 *     alpha = eps_inj / (2 E_B) evaluated from the field the right-hand side
 *     is taken of, so that the injected power sum_B Re(fh . uh*) equals
 *     eps_inj exactly at every stage;
 *   - integrating-factor SSP Runge-Kutta of order 2 or 3 (Shu-Osher form);
 *   - CFL step dt = cfl (2 pi / N) / max_i max_x |u_i| from the field at the
 *     start of the step ("CFL = 0.2", Sec. IV), capped at dt_max;
 *   - initial field: white noise, projected, dealiased, shell energies set
 *     to E0(s) ~ s^4 exp(-s^2/2), total energy init_energy.
 */
#define _GNU_SOURCE
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

int or_kc(int N) { return (N + 2) / 3 - 1; }

/* signed wavenumber of FFT index i on an N grid */
static int wavenumber(int i, int N) { return i <= N / 2 ? i : i - N; }

static int kept(int kx, int ky, int kz, int N)
{
    const int kc = or_kc(N);
    return abs(kx) <= kc && abs(ky) <= kc && abs(kz) <= kc;
}

static int in_band(long k2, double k_lo, double k_hi)
{
    return (double)k2 >= k_lo * k_lo - 1e-9 && (double)k2 <= k_hi * k_hi + 1e-9;
}

/* multiplicity of a stored mode in the full spectrum (Hermitian pairs) */
static double multiplicity(int iz, int N) { return (iz == 0 || 2 * iz == N) ? 1.0 : 2.0; }

int or_band_modes(int N, double k_lo, double k_hi)
{
    int count = 0;
    for (int ix = 0; ix < N; ++ix)
        for (int iy = 0; iy < N; ++iy)
            for (int iz = 0; iz < N; ++iz) {
                const long kx = wavenumber(ix, N), ky = wavenumber(iy, N), kz = wavenumber(iz, N);
                if (in_band(kx * kx + ky * ky + kz * kz, k_lo, k_hi)) ++count;
            }
    return count;
}

/* ---- counter-based white noise ----------------------------------------- */
/* splitmix64 (Steele, Lea & Flood 2014): the (i+1)-th output of the
 * generator seeded with `seed` is a pure function of (seed, i). */
static uint64_t splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform in (0, 1] from the top 53 bits */
static double unit_open0(uint64_t h) { return ((double)(h >> 11) + 1.0) * 0x1.0p-53; }

/* Box-Muller (cosine branch) on draws 2*counter and 2*counter+1 */
double or_white_noise(uint64_t seed, uint64_t counter)
{
    const double u1 = unit_open0(splitmix64_at(seed, 2 * counter));
    const double u2 = unit_open0(splitmix64_at(seed, 2 * counter + 1));
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* ---- spectral helpers -------------------------------------------------- */
static long spec_len(int N) { return (long)N * N * (N / 2 + 1); }

static void zero_unkept(double *uh, int N)
{
    const int H = N / 2 + 1;
    for (int ix = 0; ix < N; ++ix)
        for (int iy = 0; iy < N; ++iy)
            for (int iz = 0; iz < H; ++iz) {
                const int kx = wavenumber(ix, N), ky = wavenumber(iy, N);
                const long i = ((long)ix * N + iy) * H + iz;
                /* the Nyquist index -N/2 is never kept (kc < N/2) */
                if (!kept(kx, ky, iz, N) || 2 * ix == N || 2 * iy == N || (ix == 0 && iy == 0 && iz == 0)) {
                    uh[2 * i] = 0.0;
                    uh[2 * i + 1] = 0.0;
                }
            }
}

/* apply the Leray projector to a 3-component spectral field in place */
static void project(double *f, int N)
{
    const int H = N / 2 + 1;
    const long L = spec_len(N);
    for (int ix = 0; ix < N; ++ix)
        for (int iy = 0; iy < N; ++iy)
            for (int iz = 0; iz < H; ++iz) {
                const long i = ((long)ix * N + iy) * H + iz;
                const double k[3] = {wavenumber(ix, N), wavenumber(iy, N), iz};
                const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                if (k2 == 0.0) {
                    for (int c = 0; c < 3; ++c) f[2 * (c * L + i)] = f[2 * (c * L + i) + 1] = 0.0;
                    continue;
                }
                double kdr = 0.0, kdi = 0.0;
                for (int c = 0; c < 3; ++c) {
                    kdr += k[c] * f[2 * (c * L + i)];
                    kdi += k[c] * f[2 * (c * L + i) + 1];
                }
                for (int c = 0; c < 3; ++c) {
                    f[2 * (c * L + i)] -= k[c] * kdr / k2;
                    f[2 * (c * L + i) + 1] -= k[c] * kdi / k2;
                }
            }
}

void or_sums(const or_member *m, const double *uh, double *E, double *diss, double *EB)
{
    const int N = m->N, H = N / 2 + 1;
    const long L = spec_len(N);
    double e = 0.0, d = 0.0, eb = 0.0;
    for (int ix = 0; ix < N; ++ix)
        for (int iy = 0; iy < N; ++iy)
            for (int iz = 0; iz < H; ++iz) {
                const long i = ((long)ix * N + iy) * H + iz;
                const long kx = wavenumber(ix, N), ky = wavenumber(iy, N), kz = iz;
                const long k2 = kx * kx + ky * ky + kz * kz;
                double a2 = 0.0;
                for (int c = 0; c < 3; ++c) {
                    const double re = uh[2 * (c * L + i)], im = uh[2 * (c * L + i) + 1];
                    a2 += re * re + im * im;
                }
                const double w = multiplicity(iz, N);
                e += 0.5 * w * a2;
                d += m->nu * (double)k2 * w * a2;
                if (in_band(k2, m->k_lo, m->k_hi)) eb += 0.5 * w * a2;
            }
    if (E) *E = e;
    if (diss) *diss = d;
    if (EB) *EB = eb;
}

void or_initial_field(const or_member *m, double *uh)
{
    const int N = m->N, H = N / 2 + 1;
    const long n3 = (long)N * N * N, L = spec_len(N);
    double *u = (double *)malloc(sizeof(double) * n3);
    for (int c = 0; c < 3; ++c) {
        for (long idx = 0; idx < n3; ++idx) u[idx] = or_white_noise(m->seed, (uint64_t)c * n3 + idx);
        or_rfft3(u, uh + 2 * c * L, N);
        zero_unkept(uh + 2 * c * L, N);
    }
    free(u);
    project(uh, N);
    /* shell energies of the projected noise, shell s = round(|k|) */
    const int smax = (int)ceil(sqrt(3.0) * N / 2) + 2;
    double *shell = (double *)calloc(smax, sizeof(double));
    for (int ix = 0; ix < N; ++ix)
        for (int iy = 0; iy < N; ++iy)
            for (int iz = 0; iz < H; ++iz) {
                const long i = ((long)ix * N + iy) * H + iz;
                const long kx = wavenumber(ix, N), ky = wavenumber(iy, N), kz = iz;
                const int s = (int)lround(sqrt((double)(kx * kx + ky * ky + kz * kz)));
                for (int c = 0; c < 3; ++c) {
                    const double re = uh[2 * (c * L + i)], im = uh[2 * (c * L + i) + 1];
                    shell[s] += 0.5 * multiplicity(iz, N) * (re * re + im * im);
                }
            }
    /* target shell spectrum E0(s) = s^4 exp(-s^2/2), over occupied shells */
    double target_total = 0.0;
    for (int s = 1; s < smax; ++s)
        if (shell[s] > 0.0) target_total += pow((double)s, 4) * exp(-0.5 * s * s);
    for (int ix = 0; ix < N; ++ix)
        for (int iy = 0; iy < N; ++iy)
            for (int iz = 0; iz < H; ++iz) {
                const long i = ((long)ix * N + iy) * H + iz;
                const long kx = wavenumber(ix, N), ky = wavenumber(iy, N), kz = iz;
                const int s = (int)lround(sqrt((double)(kx * kx + ky * ky + kz * kz)));
                double f = 0.0;
                if (s > 0 && shell[s] > 0.0)
                    f = sqrt(m->init_energy * pow((double)s, 4) * exp(-0.5 * s * s) / (target_total * shell[s]));
                for (int c = 0; c < 3; ++c) {
                    uh[2 * (c * L + i)] *= f;
                    uh[2 * (c * L + i) + 1] *= f;
                }
            }
    free(shell);
}

void or_rhs(const or_member *m, const double *uh, double *F, double *nl, double *umax_out,
            double *alpha_out)
{
    const int N = m->N, H = N / 2 + 1;
    const long n3 = (long)N * N * N, L = spec_len(N);
    /* vorticity wh = i k x uh */
    double *wh = (double *)malloc(sizeof(double) * 2 * 3 * L);
    for (int ix = 0; ix < N; ++ix)
        for (int iy = 0; iy < N; ++iy)
            for (int iz = 0; iz < H; ++iz) {
                const long i = ((long)ix * N + iy) * H + iz;
                const double k[3] = {wavenumber(ix, N), wavenumber(iy, N), iz};
                for (int c = 0; c < 3; ++c) {
                    const int a = (c + 1) % 3, b = (c + 2) % 3;
                    /* (k x u)_c = k_a u_b - k_b u_a ; times i: (re, im) -> (-im, re) */
                    const double cr = k[a] * uh[2 * (b * L + i)] - k[b] * uh[2 * (a * L + i)];
                    const double ci = k[a] * uh[2 * (b * L + i) + 1] - k[b] * uh[2 * (a * L + i) + 1];
                    wh[2 * (c * L + i)] = -ci;
                    wh[2 * (c * L + i) + 1] = cr;
                }
            }
    double *u = (double *)malloc(sizeof(double) * 3 * n3);
    double *w = (double *)malloc(sizeof(double) * 3 * n3);
    for (int c = 0; c < 3; ++c) {
        or_irfft3(uh + 2 * c * L, u + c * n3, N);
        or_irfft3(wh + 2 * c * L, w + c * n3, N);
    }
    double umax = 0.0;
    double *n = (double *)malloc(sizeof(double) * 3 * n3);
    for (long p = 0; p < n3; ++p) {
        const double ux = u[p], uy = u[n3 + p], uz = u[2 * n3 + p];
        const double wx = w[p], wy = w[n3 + p], wz = w[2 * n3 + p];
        n[p] = uy * wz - uz * wy;
        n[n3 + p] = uz * wx - ux * wz;
        n[2 * n3 + p] = ux * wy - uy * wx;
        umax = fmax(umax, fmax(fabs(ux), fmax(fabs(uy), fabs(uz))));
    }
    for (int c = 0; c < 3; ++c) {
        or_rfft3(n + c * n3, F + 2 * c * L, N);
        zero_unkept(F + 2 * c * L, N);
    }
    project(F, N);
    if (nl) memcpy(nl, F, sizeof(double) * 2 * 3 * L);
    /* constant-power band forcing */
    double EB;
    or_sums(m, uh, NULL, NULL, &EB);
    const double alpha = EB > 0.0 ? exp(m->lambda) * m->eps_bar / (2.0 * EB) : 0.0;
    for (int ix = 0; ix < N; ++ix)
        for (int iy = 0; iy < N; ++iy)
            for (int iz = 0; iz < H; ++iz) {
                const long kx = wavenumber(ix, N), ky = wavenumber(iy, N), kz = iz;
                if (!in_band(kx * kx + ky * ky + kz * kz, m->k_lo, m->k_hi)) continue;
                const long i = ((long)ix * N + iy) * H + iz;
                for (int c = 0; c < 3; ++c) {
                    F[2 * (c * L + i)] += alpha * uh[2 * (c * L + i)];
                    F[2 * (c * L + i) + 1] += alpha * uh[2 * (c * L + i) + 1];
                }
            }
    if (umax_out) *umax_out = umax;
    if (alpha_out) *alpha_out = alpha;
    free(n);
    free(w);
    free(u);
    free(wh);
}

/* out = a * E(ha) x + b * E(hb) (y + dt F), E(h) = exp(-nu k^2 h), per mode.
 * x or y may be NULL (term dropped). */
static void combine(const or_member *m, double *out, double a, double ha, const double *x,
                    double b, double hb, const double *y, double dt, const double *F)
{
    const int N = m->N, H = N / 2 + 1;
    const long L = spec_len(N);
    for (int ix = 0; ix < N; ++ix)
        for (int iy = 0; iy < N; ++iy)
            for (int iz = 0; iz < H; ++iz) {
                const long i = ((long)ix * N + iy) * H + iz;
                const double kx = wavenumber(ix, N), ky = wavenumber(iy, N), kz = iz;
                const double k2 = kx * kx + ky * ky + kz * kz;
                const double ea = exp(-m->nu * k2 * ha), eb = exp(-m->nu * k2 * hb);
                for (int c = 0; c < 3; ++c)
                    for (int r = 0; r < 2; ++r) {
                        const long j = 2 * (c * L + i) + r;
                        double v = b * eb * (y[j] + dt * F[j]);
                        if (x) v += a * ea * x[j];
                        out[j] = v;
                    }
            }
}

int or_step(const or_member *m, double *uh, int nsteps, double *t, or_diag *d)
{
    const int N = m->N;
    const long L = spec_len(N);
    const size_t bytes = sizeof(double) * 2 * 3 * L;
    double *F = (double *)malloc(bytes);
    double *u1 = (double *)malloc(bytes);
    double *u2 = (double *)malloc(bytes);
    int status = 0;
    double dt = m->dt, umax = 0.0, alpha = 0.0, EB = 0.0;
    for (int s = 0; s < nsteps && status == 0; ++s) {
        or_sums(m, uh, NULL, NULL, &EB);
        if (!(EB > 0.0)) { status = -1; break; }
        or_rhs(m, uh, F, NULL, &umax, &alpha);
        if (!isfinite(umax)) { status = -2; break; }
        if (m->dt > 0.0) {
            dt = m->dt;
        } else {
            dt = m->cfl * (2.0 * M_PI / N) / umax;
            if (m->dt_max > 0.0 && dt > m->dt_max) dt = m->dt_max;
        }
        /* u1 = E(dt) (u^n + dt F(u^n)) */
        combine(m, u1, 0.0, 0.0, NULL, 1.0, dt, uh, dt, F);
        if (m->rk_order == 2) {
            /* u^{n+1} = 1/2 E(dt) u^n + 1/2 (u1 + dt F(u1)) */
            or_sums(m, u1, NULL, NULL, &EB);
            if (!(EB > 0.0)) { status = -1; break; }
            or_rhs(m, u1, F, NULL, NULL, &alpha);
            combine(m, uh, 0.5, dt, uh, 0.5, 0.0, u1, dt, F);
        } else {
            /* u2 = 3/4 E(dt/2) u^n + 1/4 E(-dt/2) (u1 + dt F(u1)) */
            or_sums(m, u1, NULL, NULL, &EB);
            if (!(EB > 0.0)) { status = -1; break; }
            or_rhs(m, u1, F, NULL, NULL, &alpha);
            combine(m, u2, 0.75, 0.5 * dt, uh, 0.25, -0.5 * dt, u1, dt, F);
            /* u^{n+1} = 1/3 E(dt) u^n + 2/3 E(dt/2) (u2 + dt F(u2)) */
            or_sums(m, u2, NULL, NULL, &EB);
            if (!(EB > 0.0)) { status = -1; break; }
            or_rhs(m, u2, F, NULL, NULL, &alpha);
            combine(m, uh, 1.0 / 3.0, dt, uh, 2.0 / 3.0, 0.5 * dt, u2, dt, F);
        }
        *t += dt;
    }
    if (d) {
        d->t = *t;
        d->dt = dt;
        or_sums(m, uh, &d->E, &d->diss, &d->EB);
        d->P = alpha * 2.0 * EB;
        d->umax = umax;
    }
    free(u2);
    free(u1);
    free(F);
    return status;
}
