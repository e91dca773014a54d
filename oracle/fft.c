/*
 * Oracle FFT: plain recursive mixed-radix Cooley-Tukey in FP64.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper's solver works on "velocity Fourier coefficients" (Sec. IV);
 * the transform pair used here is the discrete Fourier series of a
 * 2pi-periodic field sampled at x_j = 2 pi j / N.  Nothing is blocked,
 * fused or reordered: one axis at a time, one line at a time.
 */
#define _GNU_SOURCE
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Table of W_n^e = exp(sign * 2 pi i e / n), e in [0, n). */
static double *twiddle_table(int n, int sign)
{
    double *w = (double *)malloc(sizeof(double) * 2 * n);
    for (int e = 0; e < n; ++e) {
        const double a = 2.0 * M_PI * (double)e / (double)n;
        w[2 * e] = cos(a);
        w[2 * e + 1] = (double)sign * sin(a);
    }
    return w;
}

static int smallest_factor(int n)
{
    if (n % 2 == 0) return 2;
    if (n % 3 == 0) return 3;
    for (int f = 5; f * f <= n; f += 2)
        if (n % f == 0) return f;
    return n;
}

/* out[k] = sum_j in[j*stride] W_n^{jk}, k < n.  out is contiguous.
 * w is the table of the top-level length ntop; W_n^e = w[e * ntop / n]. */
static void fft_rec(const double *in, int n, int stride, double *out,
                    const double *w, int ntop)
{
    if (n == 1) {
        out[0] = in[0];
        out[1] = in[1];
        return;
    }
    const int p = smallest_factor(n);
    const int m = n / p;
    const long step = ntop / n;
    /* p decimated sub-transforms: Y_r[k] = sum_j x[p j + r] W_m^{jk} */
    for (int r = 0; r < p; ++r)
        fft_rec(in + 2 * (long)r * stride, m, stride * p, out + 2 * (long)r * m, w, ntop);
    /* combine: X[k + q m] = sum_r W_n^{r (k + q m)} Y_r[k] */
    double ybuf[2 * 64];
    double *y = p <= 64 ? ybuf : (double *)malloc(sizeof(double) * 2 * p);
    for (int k = 0; k < m; ++k) {
        for (int r = 0; r < p; ++r) {
            y[2 * r] = out[2 * (r * m + k)];
            y[2 * r + 1] = out[2 * (r * m + k) + 1];
        }
        for (int q = 0; q < p; ++q) {
            double sr = 0.0, si = 0.0;
            for (int r = 0; r < p; ++r) {
                const long e = ((long)r * (k + (long)q * m)) % n;
                const double wr = w[2 * e * step], wi = w[2 * e * step + 1];
                sr += y[2 * r] * wr - y[2 * r + 1] * wi;
                si += y[2 * r] * wi + y[2 * r + 1] * wr;
            }
            out[2 * (q * m + k)] = sr;
            out[2 * (q * m + k) + 1] = si;
        }
    }
    if (y != ybuf) free(y);
}

void or_fft1(double *data, int n, int sign)
{
    double *tmp = (double *)malloc(sizeof(double) * 2 * n);
    double *w = twiddle_table(n, sign);
    fft_rec(data, n, 1, tmp, w, n);
    memcpy(data, tmp, sizeof(double) * 2 * n);
    free(w);
    free(tmp);
}

/* Transform every line of a complex 3D array [n0][n1][n2] along one axis.
 * Lines along axis a are gathered, transformed and scattered back. */
static void fft_axis(double *c, int n0, int n1, int n2, int axis, int sign)
{
    const int len = axis == 0 ? n0 : (axis == 1 ? n1 : n2);
    const long s0 = (long)n1 * n2, s1 = n2;
    const long stride = axis == 0 ? s0 : (axis == 1 ? s1 : 1);
    const int na = axis == 0 ? n1 : n0;
    const int nb = axis == 2 ? n1 : n2;
#pragma omp parallel
    {
        double *line = (double *)malloc(sizeof(double) * 2 * len);
#pragma omp for collapse(2) schedule(static)
        for (int a = 0; a < na; ++a) {
            for (int b = 0; b < nb; ++b) {
                long base;
                if (axis == 0) base = (long)a * s1 + b;
                else if (axis == 1) base = (long)a * s0 + b;
                else base = (long)a * s0 + (long)b * s1;
                for (int j = 0; j < len; ++j) {
                    line[2 * j] = c[2 * (base + j * stride)];
                    line[2 * j + 1] = c[2 * (base + j * stride) + 1];
                }
                or_fft1(line, len, sign);
                for (int j = 0; j < len; ++j) {
                    c[2 * (base + j * stride)] = line[2 * j];
                    c[2 * (base + j * stride) + 1] = line[2 * j + 1];
                }
            }
        }
        free(line);
    }
}

void or_rfft3(const double *u, double *uh, int N)
{
    const int H = N / 2 + 1;
    const long n3 = (long)N * N * N;
    /* full complex transform of the real field, then keep kz <= N/2 */
    double *c = (double *)malloc(sizeof(double) * 2 * n3);
    for (long i = 0; i < n3; ++i) {
        c[2 * i] = u[i];
        c[2 * i + 1] = 0.0;
    }
    fft_axis(c, N, N, N, 2, -1);
    fft_axis(c, N, N, N, 1, -1);
    fft_axis(c, N, N, N, 0, -1);
    const double scale = 1.0 / (double)n3;
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y)
            for (int z = 0; z < H; ++z) {
                const long src = ((long)x * N + y) * N + z;
                const long dst = ((long)x * N + y) * H + z;
                uh[2 * dst] = c[2 * src] * scale;
                uh[2 * dst + 1] = c[2 * src + 1] * scale;
            }
    free(c);
}

void or_irfft3(const double *uh, double *u, int N)
{
    const int H = N / 2 + 1;
    const long n3 = (long)N * N * N;
    double *c = (double *)malloc(sizeof(double) * 2 * (long)N * N * H);
    memcpy(c, uh, sizeof(double) * 2 * (long)N * N * H);
    fft_axis(c, N, N, H, 0, +1);
    fft_axis(c, N, N, H, 1, +1);
    /* along z: Hermitian extension of each row, inverse, real part */
#pragma omp parallel
    {
        double *row = (double *)malloc(sizeof(double) * 2 * N);
#pragma omp for collapse(2) schedule(static)
        for (int x = 0; x < N; ++x)
            for (int y = 0; y < N; ++y) {
                const double *h = c + 2 * (((long)x * N + y) * H);
                for (int k = 0; k < N; ++k) {
                    if (k < H) {
                        row[2 * k] = h[2 * k];
                        row[2 * k + 1] = h[2 * k + 1];
                    } else {
                        row[2 * k] = h[2 * (N - k)];
                        row[2 * k + 1] = -h[2 * (N - k) + 1];
                    }
                }
                or_fft1(row, N, +1);
                double *out = u + ((long)x * N + y) * N;
                for (int z = 0; z < N; ++z) out[z] = row[2 * z];
            }
        free(row);
    }
    free(c);
    (void)n3;
}
