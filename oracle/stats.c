/*
 * Oracle velocity-gradient statistics, FP64.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * A_ij = d_j u_i; Q = -1/2 Tr A^2 and R = -1/3 Tr A^3 (Sec. V, the
 * definitions preceding the QR-PDF discussion); dissipation
 * eps = 2 nu Tr S^2 with S = (A + A^T)/2 and enstrophy omega^2 (Sec. VI).
 * [R] Histogram units: q0 = eps_norm / (2 nu_norm), i.e. <Tr S^2> of a
 * member whose mean dissipation equals eps_norm (the paper plots the QR-PDF
 * in units of <Tr S^2>, Sec. VI).  Q axis: Q/q0, R axis: R/q0^(3/2);
 * dissipation axis: eps/eps_norm; enstrophy axis: omega^2 nu_norm/eps_norm,
 * both on log10 bins.  Gradient components (Sec. VI, longitudinal and
 * transverse gradient PDFs): A_ij / sqrt(q0) on a linear axis, the three
 * longitudinal components pooled in one histogram and the six transverse
 * ones in another (isotropy).
 * [R] Bin rule: the edges are formed in FP64 and rounded to FP32; a value is
 * rounded to FP32 and lands in bin b iff edge[b] <= value < edge[b+1].
 * Values below the first edge count as underflow, at or above the last edge
 * as overflow; a non-positive value on a log axis is underflow; a
 * non-finite value goes to the nonfinite counter only.
 */
#define _GNU_SOURCE
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

int or_counts_len(const or_hist_spec *h)
{
    return h->qr_bins * h->qr_bins + 2 * h->tail_bins + 8 + (h->grad_bins > 0 ? 2 * h->grad_bins + 4 : 0);
}

static int wavenumber(int i, int N) { return i <= N / 2 ? i : i - N; }

void or_gradient(const double *uh, int N, double *A)
{
    const int H = N / 2 + 1;
    const long L = (long)N * N * H, n3 = (long)N * N * N;
    double *g = (double *)malloc(sizeof(double) * 2 * L);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            /* (d_j u_i)^ = i k_j uh_i */
            for (int ix = 0; ix < N; ++ix)
                for (int iy = 0; iy < N; ++iy)
                    for (int iz = 0; iz < H; ++iz) {
                        const long p = ((long)ix * N + iy) * H + iz;
                        const double k[3] = {wavenumber(ix, N), wavenumber(iy, N), iz};
                        const double re = uh[2 * (i * L + p)], im = uh[2 * (i * L + p) + 1];
                        g[2 * p] = -k[j] * im;
                        g[2 * p + 1] = k[j] * re;
                    }
            or_irfft3(g, A + (long)(3 * i + j) * n3, N);
        }
    free(g);
}

void or_invariants(const double *A, int N, double nu, double *Q, double *R, double *eps, double *ens)
{
    const long n3 = (long)N * N * N;
    for (long p = 0; p < n3; ++p) {
        double a[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) a[i][j] = A[(long)(3 * i + j) * n3 + p];
        double tr2 = 0.0, tr3 = 0.0, ss = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                tr2 += a[i][j] * a[j][i];
                for (int k = 0; k < 3; ++k) tr3 += a[i][j] * a[j][k] * a[k][i];
                const double s = 0.5 * (a[i][j] + a[j][i]);
                ss += s * s;
            }
        const double wx = a[2][1] - a[1][2], wy = a[0][2] - a[2][0], wz = a[1][0] - a[0][1];
        if (Q) Q[p] = -0.5 * tr2;
        if (R) R[p] = -tr3 / 3.0;
        if (eps) eps[p] = 2.0 * nu * ss;
        if (ens) ens[p] = wx * wx + wy * wy + wz * wz;
    }
}

/* edges of a linear axis [lo, hi) with n bins, FP64 rounded to FP32 */
static void linear_edges(double lo, double hi, int n, float *e)
{
    for (int b = 0; b <= n; ++b) e[b] = (float)(lo + (hi - lo) * (double)b / (double)n);
}

/* edges of a log10 axis [lo, hi) with n bins */
static void log_edges(double lo, double hi, int n, float *e)
{
    for (int b = 0; b <= n; ++b) e[b] = (float)pow(10.0, lo + (hi - lo) * (double)b / (double)n);
}

/* bin of x on edges e[0..n]: -1 underflow, n overflow (linear search) */
static int find_bin(float x, const float *e, int n)
{
    if (x < e[0]) return -1;
    if (x >= e[n]) return n;
    int b = 0;
    while (b + 1 < n && e[b + 1] <= x) ++b;
    return b;
}

/* The bin rule alone, on values already in the axis's units: axis 0 the Q
 * axis, 1 the R axis, 2 the log10 tail axis (dissipation and enstrophy),
 * 3 the gradient-component axis; out[i] = -1 underflow (and a non-positive
 * value on the log axis), n overflow, else the bin. */
void or_bin_values(const or_hist_spec *h, int axis, const float *x, long n, int *out)
{
    int nb = 0;
    float *e = NULL;
    if (axis == 0 || axis == 1 || axis == 3) {
        const double lim = axis == 0 ? h->q_lim : axis == 1 ? h->r_lim : h->grad_lim;
        nb = axis == 3 ? h->grad_bins : h->qr_bins;
        e = (float *)malloc(sizeof(float) * (nb + 1));
        linear_edges(-lim, lim, nb, e);
    } else {
        nb = h->tail_bins;
        e = (float *)malloc(sizeof(float) * (nb + 1));
        log_edges(h->tail_lo, h->tail_hi, nb, e);
    }
    for (long i = 0; i < n; ++i) out[i] = (axis == 2 && !(x[i] > 0.0f)) ? -1 : find_bin(x[i], e, nb);
    free(e);
}

void or_gradient_stats(const double *uh, int N, double nu, const or_hist_spec *h, uint64_t *counts,
                       double *moments)
{
    const long n3 = (long)N * N * N;
    double *A = (double *)malloc(sizeof(double) * 9 * n3);
    double *Q = (double *)malloc(sizeof(double) * n3);
    double *R = (double *)malloc(sizeof(double) * n3);
    double *eps = (double *)malloc(sizeof(double) * n3);
    double *ens = (double *)malloc(sizeof(double) * n3);
    or_gradient(uh, N, A);
    or_invariants(A, N, nu, Q, R, eps, ens);

    const int nq = h->qr_bins, nt = h->tail_bins;
    float *eq = (float *)malloc(sizeof(float) * (nq + 1));
    float *er = (float *)malloc(sizeof(float) * (nq + 1));
    float *et = (float *)malloc(sizeof(float) * (nt + 1));
    linear_edges(-h->q_lim, h->q_lim, nq, eq);
    linear_edges(-h->r_lim, h->r_lim, nq, er);
    log_edges(h->tail_lo, h->tail_hi, nt, et);
    const double q0 = h->eps_norm / (2.0 * h->nu_norm);
    const double r0 = pow(q0, 1.5);
    uint64_t *qr = counts, *he = counts + nq * nq, *hw = he + nt, *ctr = hw + nt;
    const int ng = h->grad_bins;
    float *eg = NULL;
    if (ng > 0) {
        eg = (float *)malloc(sizeof(float) * (ng + 1));
        linear_edges(-h->grad_lim, h->grad_lim, ng, eg);
    }
    uint64_t *hl = ctr + 8, *ht = hl + ng, *gctr = ht + ng;
    const double g0 = sqrt(q0);

    for (long p = 0; p < n3; ++p) {
        const double vals[4] = {Q[p] / q0, R[p] / r0, eps[p] / h->eps_norm, ens[p] * h->nu_norm / h->eps_norm};
        int finite = 1;
        for (int v = 0; v < 4; ++v) finite &= isfinite(vals[v]) ? 1 : 0;
        ctr[6] += 1;
        if (!finite) { ctr[5] += 1; continue; }
        const int bq = find_bin((float)vals[0], eq, nq), br = find_bin((float)vals[1], er, nq);
        if (bq >= 0 && bq < nq && br >= 0 && br < nq) qr[(long)bq * nq + br] += 1;
        else ctr[0] += 1;
        for (int t = 0; t < 2; ++t) {
            const float x = (float)vals[2 + t];
            uint64_t *hist = t == 0 ? he : hw;
            const int b = x > 0.0f ? find_bin(x, et, nt) : -1;
            if (b < 0) ctr[1 + 2 * t] += 1;
            else if (b >= nt) ctr[2 + 2 * t] += 1;
            else hist[b] += 1;
        }
        /* gradient components: c = 3 i + j, longitudinal iff i == j */
        for (int c = 0; ng > 0 && c < 9; ++c) {
            const int lon = c % 4 == 0;
            const int b = find_bin((float)(A[(long)c * n3 + p] / g0), eg, ng);
            uint64_t *hist = lon ? hl : ht;
            if (b < 0) gctr[lon ? 0 : 2] += 1;
            else if (b >= ng) gctr[lon ? 1 : 3] += 1;
            else hist[b] += 1;
        }
    }
    free(eg);
    /* moments: sum A_c^p, p in {2,3,4,6}, c row-major; then sums of
     * Q, R, eps, omega^2, Q^2, R^2, eps^2, omega^4 */
    for (long p = 0; p < n3; ++p) {
        for (int c = 0; c < 9; ++c) {
            const double a = A[(long)c * n3 + p], a2 = a * a;
            moments[4 * c + 0] += a2;
            moments[4 * c + 1] += a2 * a;
            moments[4 * c + 2] += a2 * a2;
            moments[4 * c + 3] += a2 * a2 * a2;
        }
        moments[36] += Q[p];
        moments[37] += R[p];
        moments[38] += eps[p];
        moments[39] += ens[p];
        moments[40] += Q[p] * Q[p];
        moments[41] += R[p] * R[p];
        moments[42] += eps[p] * eps[p];
        moments[43] += ens[p] * ens[p];
    }
    free(et);
    free(er);
    free(eq);
    free(ens);
    free(eps);
    free(R);
    free(Q);
    free(A);
}
