// Scaling-exponent theory around the mixture (Secs. III, V, VII).
//
//  - ens_lambda_weights: member weights for a general zeta_p family.  The
//    cumulant generating function of lambda is K(t; Z) = (t - zeta_3t) Z
//    (Sec. III, Eq. exponents_KZ_1); P(lambda; Z) follows from the inverse
//    two-sided Laplace transform of exp K, evaluated at imaginary t and
//    Fourier-transformed (Sec. VII), here on the device in FP64 on a uniform
//    lambda grid, then integrated over each member's lambda bin.  For the
//    log-Poisson family exp K is the transform of a shifted Poisson lattice
//    and the masses are summed exactly.
//  - ens_nelkin_exponents / ens_ratio_exponents: rho_m = m - zeta_{m+rho_m}
//    (Sec. III, Eq. nelkin_rhom) and the predicted R_lambda exponents of
//    skewness, flatness and hyper-flatness (Sec. VII).
//  - ens_scale_gap: Z for a target R_lambda from the members' R_lambda with a
//    constant C_eps (Sec. V, Eq. Re_definition and Eq. Rlambda_Z_relation).
#include "../../include/ens.h"

#include <cmath>

namespace {

constexpr int kGrid = ENS_LAMBDA_GRID;      // power of two
constexpr double kGridLo = ENS_LAMBDA_GRID_LO, kGridHi = ENS_LAMBDA_GRID_HI;
constexpr double kPi = 3.14159265358979323846;
constexpr int kFftThreads = 1024;

__host__ __device__ double zeta_real(const ens_zeta_spec &z, double p)
{
    switch (z.kind) {
    case ENS_ZETA_QUADRATIC: return p / 3.0 - z.c * (p * p - 3.0 * p) / 2.0;
    case ENS_ZETA_LOGPOISSON: return p / 9.0 + z.C0 * (1.0 - pow(z.beta, p / 3.0));
    default: return (1.0 + 3.0 * z.beta) * p / (3.0 * (1.0 + z.beta * p));
    }
}

// point mass of saturating exponents: exp(-zeta_inf Z) at lambda = Z
__host__ __device__ double atom_mass(const ens_zeta_spec &z, double Zg)
{
    if (z.kind != ENS_ZETA_RATIONAL) return 0.0;
    return exp(-(1.0 + 3.0 * z.beta) / (3.0 * z.beta) * Zg);
}

// K(i s; Z) = (i s - zeta(3 i s)) Z as (re, im)
__device__ double2 K_imag(const ens_zeta_spec &z, double Zg, double s)
{
    if (z.kind == ENS_ZETA_QUADRATIC)   // 9 c (t^2 - t) Z / 2 at t = i s
        return make_double2(-4.5 * z.c * Zg * s * s, -4.5 * z.c * Zg * s);
    // rational: zeta(3t) = (1 + 3b) t / (1 + 3b t); at t = i s multiply by
    // the conjugate (1 - 3b i s) / (1 + 9 b^2 s^2)
    const double b3 = 3.0 * z.beta, q = (1.0 + 3.0 * z.beta) * s / (1.0 + b3 * b3 * s * s);
    return make_double2(-q * b3 * s * Zg, (s - q) * Zg);
}

// phi'_k = (exp(K(i s_k)) - m_atom exp(i s_k Z)) exp(-i s_k l_0),
// s_k = 2 pi f_k / (n dl), f_k the signed frequency of index k
__global__ void k_char_fn(ens_zeta_spec z, double Zg, double2 *phi)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kGrid) return;
    const double dl = (kGridHi - kGridLo) / kGrid;
    const int f = k < kGrid / 2 ? k : k - kGrid;
    const double s = 2.0 * kPi * f / (kGrid * dl);
    const double2 K = K_imag(z, Zg, s);
    const double m = exp(K.x);
    double sn, cs;
    sincos(K.y, &sn, &cs);
    double re = m * cs, im = m * sn;
    const double ma = atom_mass(z, Zg);
    if (ma > 0.0) {
        sincos(s * Zg, &sn, &cs);
        re -= ma * cs;
        im -= ma * sn;
    }
    sincos(-s * kGridLo, &sn, &cs);
    phi[k] = make_double2(re * cs - im * sn, re * sn + im * cs);
}

// Forward FFT of phi' (radix-2 Stockham autosort, natural order out), one
// CTA ping-ponging between a and b through L2; P_j = Re(...)_j / (n dl)
__global__ void __launch_bounds__(kFftThreads) k_fft_pdf(double2 *a, double2 *b, double *P)
{
    constexpr int half = kGrid / 2;
    double2 *src = a, *dst = b;
    for (int ns = 1; ns < kGrid; ns <<= 1) {
        for (int j = threadIdx.x; j < half; j += kFftThreads) {
            const double2 v0 = src[j], x1 = src[j + half];
            const int r = j & (ns - 1);
            double sn, cs;
            sincospi(-(double)r / ns, &sn, &cs);
            const double2 v1 = make_double2(x1.x * cs - x1.y * sn, x1.x * sn + x1.y * cs);
            const int d = (j - r) * 2 + r;       // (j / ns) * 2 ns + j mod ns
            dst[d] = make_double2(v0.x + v1.x, v0.y + v1.y);
            dst[d + ns] = make_double2(v0.x - v1.x, v0.y - v1.y);
        }
        __syncthreads();
        double2 *t = src;
        src = dst;
        dst = t;
    }
    for (int j = threadIdx.x; j < kGrid; j += kFftThreads) P[j] = src[j].x / (kGridHi - kGridLo);
}

__device__ void member_bin(const double *lam, int n, int i, double *lo, double *hi, int *mult)
{
    const double li = lam[i];
    double prev = -INFINITY, next = INFINITY;
    int mu = 0;
    for (int j = 0; j < n; ++j) {
        const double lj = lam[j];
        if (lj == li) ++mu;
        else if (lj < li && lj > prev) prev = lj;
        else if (lj > li && lj < next) next = lj;
    }
    if (prev == -INFINITY && next == INFINITY) {
        *lo = -INFINITY;
        *hi = INFINITY;
    } else {
        *lo = prev == -INFINITY ? li - 0.5 * (next - li) : 0.5 * (prev + li);
        *hi = next == INFINITY ? li + 0.5 * (li - prev) : 0.5 * (li + next);
    }
    *mult = mu;
}

__device__ double grid_interp(const double *P, double x)
{
    const double dl = (kGridHi - kGridLo) / kGrid;
    const double u = (x - kGridLo) / dl;
    const int j = (int)floor(u);
    if (j >= kGrid - 1) return P[kGrid - 1];
    if (j < 0) return P[0];
    const double t = u - j;
    return P[j] * (1.0 - t) + P[j + 1] * t;
}

// trapezoid integral of the grid density over each member's bin, the bin
// ends interpolated linearly, plus a point mass at atom_at
__global__ void k_bin_integrate(const double *P, const double *lam, int n, double atom_at, double atom, double *w)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double lo, hi;
    int mult;
    member_bin(lam, n, i, &lo, &hi, &mult);
    const double dl = (kGridHi - kGridLo) / kGrid;
    const double a = fmax(lo, kGridLo), b = fmin(hi, kGridLo + (kGrid - 1) * dl);
    double s = 0.0;
    if (b > a) {
        double x0 = a, y0 = grid_interp(P, a);
        for (int j = max(0, (int)floor((a - kGridLo) / dl)); j < kGrid; ++j) {
            const double x = kGridLo + j * dl;
            if (x <= a) continue;
            if (x >= b) break;
            s += 0.5 * (y0 + P[j]) * (x - x0);
            x0 = x;
            y0 = P[j];
        }
        s += 0.5 * (y0 + grid_interp(P, b)) * (b - x0);
    }
    if (atom > 0.0 && lo <= atom_at && atom_at < hi) s += atom;
    w[i] = s / mult;
}

// exact masses of lambda = 2Z/3 + k ln(beta), k ~ Poisson(C0 Z)
__global__ void k_logpoisson(ens_zeta_spec z, double Zg, const double *lam, int n, double *w)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double lo, hi;
    int mult;
    member_bin(lam, n, i, &lo, &hi, &mult);
    const double mu = z.C0 * Zg;
    double logp = -mu, s = 0.0;
    for (int k = 0; k < 400; ++k) {
        if (k > 0) logp += log(mu) - log((double)k);
        const double lk = 2.0 * Zg / 3.0 + k * log(z.beta);
        if (lo <= lk && lk < hi) s += exp(logp);
    }
    w[i] = s / mult;
}

bool valid_spec(const ens_zeta_spec &z)
{
    switch (z.kind) {
    case ENS_ZETA_QUADRATIC: return std::isfinite(z.c) && z.c >= 0.0;
    case ENS_ZETA_LOGPOISSON: return z.beta > 0.0 && z.beta < 1.0 && z.C0 > 0.0 && std::isfinite(z.C0);
    case ENS_ZETA_RATIONAL: return z.beta > 0.0 && std::isfinite(z.beta);
    default: return false;
    }
}

// device scratch of one inversion: phi and its ping-pong partner, P, then
// lambdas and weights
ens_status invert(const ens_zeta_spec &z, double Zg, cudaStream_t s, void *d)
{
    double2 *a = (double2 *)d, *b = a + kGrid;
    double *P = (double *)(b + kGrid);
    k_char_fn<<<kGrid / 256, 256, 0, s>>>(z, Zg, a);
    k_fft_pdf<<<1, kFftThreads, 0, s>>>(a, b, P);
    return cudaGetLastError() == cudaSuccess ? ENS_OK : ENS_ECUDA;
}

constexpr size_t kInvBytes = sizeof(double2) * 2 * kGrid + sizeof(double) * kGrid;

}  // namespace

extern "C" {

ens_status ens_lambda_weights(const ens_zeta_spec *z, double Z, int n, const double *lambdas, double *weights,
                              double *covered, void *stream)
{
    if (!z || n <= 0 || !lambdas || !weights || !(Z > 0.0) || !std::isfinite(Z) || !valid_spec(*z))
        return ENS_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(lambdas[i])) return ENS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    void *d = nullptr;
    if (cudaMallocAsync(&d, kInvBytes + sizeof(double) * 2 * (size_t)n, s) != cudaSuccess) {
        cudaGetLastError();
        return ENS_ENOMEM;
    }
    const double *P = (const double *)((double2 *)d + 2 * kGrid);
    double *dlam = (double *)((char *)d + kInvBytes), *dw = dlam + n;
    ens_status st = ENS_OK;
    if (cudaMemcpyAsync(dlam, lambdas, sizeof(double) * n, cudaMemcpyHostToDevice, s) != cudaSuccess) st = ENS_ECUDA;
    if (st == ENS_OK) {
        if (z->kind == ENS_ZETA_LOGPOISSON) {
            k_logpoisson<<<(n + 63) / 64, 64, 0, s>>>(*z, Z, dlam, n, dw);
        } else {
            st = invert(*z, Z, s, d);
            k_bin_integrate<<<(n + 63) / 64, 64, 0, s>>>(P, dlam, n, Z, atom_mass(*z, Z), dw);
        }
        if (st == ENS_OK && (cudaGetLastError() != cudaSuccess ||
                             cudaMemcpyAsync(weights, dw, sizeof(double) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess))
            st = ENS_ECUDA;
    }
    cudaFreeAsync(d, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) st = ENS_ECUDA;
    if (st == ENS_OK && covered) {
        double t = 0.0;
        for (int i = 0; i < n; ++i) t += weights[i];
        *covered = t;
    }
    return st;
}

ens_status ens_lambda_pdf(const ens_zeta_spec *z, double Z, double *pdf, void *stream)
{
    if (!z || !pdf || !(Z > 0.0) || !std::isfinite(Z) || !valid_spec(*z) || z->kind == ENS_ZETA_LOGPOISSON)
        return ENS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    void *d = nullptr;
    if (cudaMallocAsync(&d, kInvBytes, s) != cudaSuccess) {
        cudaGetLastError();
        return ENS_ENOMEM;
    }
    ens_status st = invert(*z, Z, s, d);
    if (st == ENS_OK && cudaMemcpyAsync(pdf, (double2 *)d + 2 * kGrid, sizeof(double) * kGrid,
                                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = ENS_ECUDA;
    cudaFreeAsync(d, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) st = ENS_ECUDA;
    return st;
}

ens_status ens_nelkin_exponents(const ens_zeta_spec *z, int nm, const double *m, double *rho)
{
    if (!z || nm <= 0 || !m || !rho || !valid_spec(*z)) return ENS_EINVAL;
    for (int q = 0; q < nm; ++q) {
        if (!std::isfinite(m[q])) return ENS_EINVAL;
        auto f = [&](double r) { return r - m[q] + zeta_real(*z, m[q] + r); };
        double lo = -10.0, hi = 10.0;
        // the rational form has a pole at p = -1/beta: keep the bracket above it
        if (z->kind == ENS_ZETA_RATIONAL) lo = std::fmax(lo, -m[q] - 1.0 / z->beta + 1e-9);
        if (!(f(lo) < 0.0 && f(hi) > 0.0)) return ENS_EINVAL;
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (f(mid) < 0.0) lo = mid;
            else hi = mid;
        }
        rho[q] = 0.5 * (lo + hi);
    }
    return ENS_OK;
}

ens_status ens_ratio_exponents(const ens_zeta_spec *z, double *out)
{
    if (!out) return ENS_EINVAL;
    const double m[4] = {2, 3, 4, 6};
    double r[4];
    const ens_status s = ens_nelkin_exponents(z, 4, m, r);
    if (s != ENS_OK) return s;
    out[0] = 2 * r[1] - 3 * r[0];
    out[1] = 2 * r[2] - 4 * r[0];
    out[2] = 2 * r[3] - 6 * r[0];
    return ENS_OK;
}

ens_status ens_scale_gap(int n, const double *lambdas, const double *rlambda, double R_ref, double *Z, double *R0)
{
    if (n <= 0 || !lambdas || !rlambda || !(R_ref > 0.0) || !Z) return ENS_EINVAL;
    double s = 0.0;
    int k = 0;
    for (int i = 0; i < n; ++i) {
        if (!(lambdas[i] >= 0.0)) continue;
        if (!(rlambda[i] > 0.0) || !std::isfinite(rlambda[i])) return ENS_EINVAL;
        s += std::log(rlambda[i]) - lambdas[i] / 6.0;
        ++k;
    }
    if (k == 0) return ENS_EINVAL;
    const double r0 = std::exp(s / k);
    if (R0) *R0 = r0;
    *Z = 1.5 * std::log(R_ref / r0);
    return ENS_OK;
}

}  // extern "C"
