"""Oracle lambda weights and ensemble mixture, FP64 (numpy + math.erf).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The ensemble hypothesis (Sec. II, Eq. ensemble_hypothesis) writes a high-Reynolds-number average as
an integral over the injection-rate parameter lambda with weight P(lambda; Z).
For the quadratic scaling exponents zeta_p = p/3 - c (p^2 - 3p)/2 (Sec. IV, Eq. quadratic_scaling_exponents),
K(t; Z) = 9 c (t^2 - t) Z / 2 (Sec. IV) and P is Gaussian with mean
-9cZ/2 and variance 9cZ (Sec. IV, Eq. gaussian_lambda_pdf).  Each member owns a lambda bin and its
weight is the integral of P over that bin (Sec. IV, after Eq. gaussian_lambda_pdf); any
average is then a weighted sum over members, e.g. PDFs (Sec. II, Eq.
pdf_superposition) and the skewness prediction (Sec. VII).

Readings [R] where the paper is silent:
  - bin edges are midpoints between neighbouring distinct lambda values; the
    outer edges lie half a neighbour spacing beyond the extreme members; a
    single member's bin is the whole line;
  - members with equal lambda share their bin's mass equally;
  - weights are renormalised to sum to one by default; the raw covered mass
    is returned alongside;
  - Z = 0 is the delta distribution at lambda = 0 (Sec. VII).
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------------------
# lambda distributions
# ---------------------------------------------------------------------------
def zeta_quadratic(p, c=0.023):
    """Log-normal scaling exponents, Sec. IV, Eq. quadratic_scaling_exponents."""
    return p / 3.0 - c * (p * p - 3.0 * p) / 2.0


def K_from_zeta(t, Z, zeta):
    """Cumulant generating function from Sec. III, Eq. exponents_KZ_1: K(p/3; Z) = (p/3 - zeta_p) Z."""
    return (t - zeta(3.0 * t)) * Z


def gauss_params(c, Z):
    """Mean and standard deviation of P(lambda; Z), Sec. IV, Eq. gaussian_lambda_pdf."""
    return -4.5 * c * Z, math.sqrt(9.0 * c * Z)


def gauss_pdf(lam, c, Z):
    """P(lambda; Z) of Sec. IV, Eq. gaussian_lambda_pdf, written out."""
    lam = np.asarray(lam, dtype=np.float64)
    return np.exp(-(lam + 9.0 * c * Z / 2.0) ** 2 / (18.0 * c * Z)) / math.sqrt(18.0 * math.pi * c * Z)


def _norm_cdf(x):
    """Standard normal CDF, accurate in both tails."""
    if x == math.inf:
        return 1.0
    if x == -math.inf:
        return 0.0
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


def _norm_sf(x):
    """Standard normal upper tail 1 - CDF."""
    if x == math.inf:
        return 0.0
    if x == -math.inf:
        return 1.0
    return 0.5 * math.erfc(x / math.sqrt(2.0))


def normal_interval_mass(a, b, mu, sigma):
    """Mass of N(mu, sigma^2) on [a, b]; differences taken on the tail
    closer to the interval so that tiny masses keep their digits."""
    za, zb = (a - mu) / sigma, (b - mu) / sigma
    if za >= 0.0:
        return _norm_sf(za) - _norm_sf(zb)
    return _norm_cdf(zb) - _norm_cdf(za)


def truncated_gauss_params(c, Z):
    """Appendix, Eq. truncated_gaussian: P = N exp(-(lambda-mu)^2 / (18 c Z)) Theta(Z - lambda).
    Returns (mu, sigma, cut) with mu solved in FP64 so that int P e^lambda = 1.
    Normalisation: N = 1 / (sigma sqrt(2 pi) Phi((Z - mu)/sigma))."""
    sigma = math.sqrt(9.0 * c * Z)

    def constraint(mu):
        # int_{-inf}^{Z} e^l N(l; mu, s^2) dl / Phi((Z - mu)/s) - 1, in logs
        a = mu + 0.5 * sigma * sigma
        return a + math.log(_norm_cdf((Z - mu - sigma * sigma) / sigma)) - math.log(
            _norm_cdf((Z - mu) / sigma))

    lo, hi = -4.5 * c * Z - 10.0 * sigma - 1.0, 10.0
    flo, fhi = constraint(lo), constraint(hi)
    assert flo < 0.0 < fhi
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        f = constraint(mid)
        if f < 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi), sigma, Z


def lambda_pdf_from_K(K, lam_grid, atom=None):
    """Numerical inverse two-sided Laplace transform (Sec. VII): evaluate
    exp(K(i s)) (the characteristic function) and Fourier-transform it.
    K must accept complex arguments.  Returns P on lam_grid (uniform).
    atom = (position, mass): a point mass known in closed form, removed from
    the characteristic function before the transform (so that it does not
    ring across the grid); the returned P is then the continuous part."""
    lam = np.asarray(lam_grid, dtype=np.float64)
    n = lam.size
    dl = lam[1] - lam[0]
    s = 2.0 * math.pi * np.fft.fftfreq(n, d=dl)
    phi = np.exp(np.array([K(1j * si) for si in s], dtype=np.complex128))
    if atom is not None:
        phi = phi - atom[1] * np.exp(1j * s * atom[0])
    # P(l_j) = 1/(2 pi) int ds exp(-i s l_j) phi(s)
    #        ~ (1/(n dl)) sum_k exp(-i s_k l_0) phi(s_k) exp(-2 pi i k j / n): a forward DFT
    P = np.real(np.fft.fft(phi * np.exp(-1j * s * lam[0]))) / (n * dl)
    return P


# ---------------------------------------------------------------------------
# lambda bins and member weights
# ---------------------------------------------------------------------------
def lambda_bins(lams):
    """Per-member bin [lo, hi] and the multiplicity of its lambda value."""
    lams = np.asarray(lams, dtype=np.float64)
    vals = np.unique(lams)
    if vals.size == 1:
        edges = np.array([-math.inf, math.inf])
    else:
        mids = 0.5 * (vals[1:] + vals[:-1])
        edges = np.concatenate(([vals[0] - 0.5 * (vals[1] - vals[0])], mids,
                                [vals[-1] + 0.5 * (vals[-1] - vals[-2])]))
    lo = np.empty_like(lams)
    hi = np.empty_like(lams)
    mult = np.empty_like(lams)
    for i, l in enumerate(lams):
        j = int(np.searchsorted(vals, l))
        lo[i], hi[i] = edges[j], edges[j + 1]
        mult[i] = np.count_nonzero(lams == l)
    return lo, hi, mult


def member_weights(lams, kind="gauss_paper", c=0.023, Z=1.0, mu=0.0, sigma=1.0, user=None,
                   renormalize=True):
    """Bin masses w_i of the members; returns (w, covered_mass).

    kind: 'gauss_paper' (Eq. gaussian_lambda_pdf with c, Z), 'gauss'
    (mu, sigma), 'trunc_gauss' (Appendix, c, Z) or 'user' (given weights)."""
    lams = np.asarray(lams, dtype=np.float64)
    lo, hi, mult = lambda_bins(lams)
    w = np.zeros_like(lams)
    if kind == "user":
        w = np.asarray(user, dtype=np.float64).copy()
    elif kind == "gauss_paper" and Z == 0.0:
        # P(lambda; 0) = delta(lambda): the whole mass sits in the bin holding 0
        for i in range(lams.size):
            if lo[i] <= 0.0 < hi[i]:
                w[i] = 1.0 / mult[i]
    elif kind in ("gauss_paper", "gauss"):
        m, s = gauss_params(c, Z) if kind == "gauss_paper" else (mu, sigma)
        for i in range(lams.size):
            w[i] = normal_interval_mass(lo[i], hi[i], m, s) / mult[i]
    elif kind == "trunc_gauss":
        m, s, cut = truncated_gauss_params(c, Z)
        norm = _norm_cdf((cut - m) / s)
        for i in range(lams.size):
            a, b = lo[i], min(hi[i], cut)
            w[i] = (normal_interval_mass(a, b, m, s) / norm / mult[i]) if b > a else 0.0
    else:
        raise ValueError(kind)
    covered = float(w.sum())
    if renormalize and covered > 0.0:
        w = w / covered
    return w, covered


# ---------------------------------------------------------------------------
# mixture of member statistics
# ---------------------------------------------------------------------------
def mix_counts(counts, weights, h):
    """Weighted PDFs from per-member histogram counts (Sec. II, Eq. pdf_superposition, discretised):
    PDF_mix(b) = sum_i w_i h_i(b) / (n_i db), n_i = all points of member i.
    counts: [n_members, counts_len] (layout of oracle.HistSpec).
    Returns (pdf_qr [nq, nq], pdf_eps [nt], pdf_ens [nt]) per unit of the
    bin coordinates (Q/q0, R/q0^1.5; log10 of the tail variables)."""
    counts = np.asarray(counts, dtype=np.float64)
    nq, nt = h.qr_bins, h.tail_bins
    npts = counts[:, nq * nq + 2 * nt + 6]
    frac = counts / npts[:, None]
    mix = (np.asarray(weights)[:, None] * frac).sum(axis=0)
    dq = 2.0 * h.q_lim / nq
    dr = 2.0 * h.r_lim / nq
    dl = (h.tail_hi - h.tail_lo) / nt
    qr = mix[: nq * nq].reshape(nq, nq) / (dq * dr)
    e = mix[nq * nq: nq * nq + nt] / dl
    w = mix[nq * nq + nt: nq * nq + 2 * nt] / dl
    return qr, e, w


def mix_gradient_pdfs(counts, weights, h):
    """Mixed PDFs of the longitudinal and transverse gradient components
    (Sec. VI, gradient PDFs; Sec. II, Eq. pdf_superposition, discretised) in
    units of A/sqrt(q0): every grid point contributes 3 longitudinal and 6
    transverse samples, so PDF(b) = sum_i w_i h_i(b) / (k n_i db), k = 3, 6."""
    counts = np.asarray(counts, dtype=np.float64)
    nq, nt, ng = h.qr_bins, h.tail_bins, h.grad_bins
    off = nq * nq + 2 * nt
    npts = counts[:, off + 6]
    db = 2.0 * h.grad_lim / ng
    w = np.asarray(weights, dtype=np.float64)[:, None]
    lon = (w * counts[:, off + 8: off + 8 + ng] / npts[:, None]).sum(axis=0) / (3.0 * db)
    tra = (w * counts[:, off + 8 + ng: off + 8 + 2 * ng] / npts[:, None]).sum(axis=0) / (6.0 * db)
    return lon, tra


def mix_moments(moments, npoints, weights):
    """<X^p>_mix = sum_i w_i <X^p>_i (Sec. II, Eq. ensemble_hypothesis with X a power)."""
    moments = np.asarray(moments, dtype=np.float64)
    per = moments / np.asarray(npoints, dtype=np.float64)[:, None]
    return (np.asarray(weights)[:, None] * per).sum(axis=0)


LONGITUDINAL = (0, 4, 8)          # A_11, A_22, A_33 (row-major index)
TRANSVERSE = (1, 2, 3, 5, 6, 7)


def gradient_moment_ratios(mixed):
    """Skewness, flatness and hyper-flatness of gradient components from
    mixed moments (Sec. VII, Eq. def_skewness_flatness and the skewness
    prediction that follows it), isotropy-averaged over the three
    longitudinal and six transverse components.  mixed: the 48 mixed
    moment averages (layout of the stats moments)."""
    def avg(comps, p):
        idx = {2: 0, 3: 1, 4: 2, 6: 3}[p]
        return float(np.mean([mixed[4 * c + idx] for c in comps]))
    L2, L3, L4, L6 = (avg(LONGITUDINAL, p) for p in (2, 3, 4, 6))
    T2, T4, T6 = (avg(TRANSVERSE, p) for p in (2, 4, 6))
    return {"S_long": L3 / L2 ** 1.5, "F_long": L4 / L2 ** 2, "F_trans": T4 / T2 ** 2,
            "H_long": L6 / L2 ** 3, "H_trans": T6 / T2 ** 3}


def member_contributions(counts, weights, h, which="eps"):
    """Per-member contribution w_i h_i(b)/n_i to each tail bin (Sec. VII,
    choice of the lambda range): [n_members, nt]."""
    counts = np.asarray(counts, dtype=np.float64)
    nq, nt = h.qr_bins, h.tail_bins
    npts = counts[:, nq * nq + 2 * nt + 6]
    off = nq * nq + (0 if which == "eps" else nt)
    return np.asarray(weights)[:, None] * counts[:, off:off + nt] / npts[:, None]


def hellinger(p, q):
    """Hellinger distance between two discrete distributions (each
    normalised to unit sum here)."""
    p = np.asarray(p, dtype=np.float64).ravel()
    q = np.asarray(q, dtype=np.float64).ravel()
    p = p / p.sum()
    q = q / q.sum()
    return math.sqrt(max(0.0, 1.0 - float(np.sum(np.sqrt(p * q)))))


def cost_ratio(R_ref, R_ens, n):
    """Sec. VI, cost estimate: Cost_DNS / Cost_ens ~ (R_ref / R_ens)^5 / n."""
    return (R_ref / R_ens) ** 5 / n


def Z_from_Rlambda(R_ref, R_ens):
    """Sec. V, Eq. Rlambda_Z_relation: R_ref ~ exp(2Z/3) with the constant fixed at Z = 0."""
    return 1.5 * math.log(R_ref / R_ens)


def fit_R0(lams, rlambda):
    """Constant-C_eps fit over the members with lambda >= 0 (Sec. V): with
    Re = C_eps^(-1/3) nu^-1 (eps L^4)^(1/3) (Eq. Re_definition) and
    R_lambda^2 ~ Re, a member's R_lambda scales as exp(lambda/6); the fit
    of ln R_lambda = ln R0 + lambda/6 gives R0, the central value."""
    sel = [(l, r) for l, r in zip(lams, rlambda) if l >= 0.0]
    return math.exp(sum(math.log(r) - l / 6.0 for l, r in sel) / len(sel))


def scale_gap(lams, rlambda, R_ref):
    """Z for a target R_lambda from the fitted central value."""
    return Z_from_Rlambda(R_ref, fit_R0(lams, rlambda))


# ---------------------------------------------------------------------------
# general scaling exponents (Sec. III / Sec. VII): zeta families and weights
# ---------------------------------------------------------------------------
def zeta_logpoisson(p, beta=2.0 / 3.0, C0=2.0):
    """Log-Poisson exponents, one of the literature parameterizations the
    paper points to (Sec. III): zeta_p = p/9 + C0 (1 - beta^(p/3))."""
    return p / 9.0 + C0 * (1.0 - beta ** (p / 3.0))


def zeta_rational(p, beta=0.05):
    """Saturating rational exponents zeta_p = (1 + 3 beta) p / (3 (1 + beta p))
    (Yakhot's mean-field form; zeta_3 = 1, zeta_p -> (1 + 3 beta)/(3 beta)).
    A saturating family of the kind the paper inverts numerically (Sec. VII,
    choice of zeta_p; Appendix, saturation gives lambda_max(Z) = Z)."""
    return (1.0 + 3.0 * beta) * p / (3.0 * (1.0 + beta * p))


def saturation_atom(zeta_inf, Z):
    """Saturating exponents, zeta_p -> zeta_inf: K(t; Z) - t Z = -zeta_3t Z
    tends to -zeta_inf Z as t -> infinity, so P(lambda; Z) holds a point mass
    exp(-zeta_inf Z) at lambda_max = Z (the Appendix's saturation argument
    carried one step further).  Returns (position, mass)."""
    return Z, math.exp(-zeta_inf * Z)


def nelkin_rho(m, zeta):
    """Gradient-moment exponent from the Nelkin relation rho_m = m - zeta_{m + rho_m}
    (Sec. III, Eq. nelkin_rhom), solved by bisection."""
    f = lambda r: r - m + zeta(m + r)
    lo, hi = -10.0, 10.0
    assert f(lo) < 0 < f(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) < 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def ratio_exponents(zeta):
    """Predicted R_lambda exponents of skewness, flatness and hyper-flatness
    (Sec. VII): 2 rho3 - 3 rho2, 2 rho4 - 4 rho2, 2 rho6 - 6 rho2."""
    r = {m: nelkin_rho(m, zeta) for m in (2, 3, 4, 6)}
    return 2 * r[3] - 3 * r[2], 2 * r[4] - 4 * r[2], 2 * r[6] - 6 * r[2]


LAMBDA_GRID = (-30.0, 30.0, 65536)     # lo, hi (exclusive), points


def weights_numeric(lams, K, Z, grid_lo=LAMBDA_GRID[0], grid_hi=LAMBDA_GRID[1], n=LAMBDA_GRID[2], atom=None):
    """Member bin masses of the lambda distribution whose cumulant generating
    function is K(t; Z) (Sec. III, Eq. cumulant_generating_function), by the
    numerical inverse two-sided Laplace transform (Sec. VII) on a uniform
    grid and trapezoid integration over each member's bin.  atom =
    (position, mass) of a known point mass: removed before the transform and
    added to the bin that holds it (lo <= position < hi)."""
    grid = np.linspace(grid_lo, grid_hi, n, endpoint=False)
    P = lambda_pdf_from_K(lambda t: K(t, Z), grid, atom)
    lo, hi, mult = lambda_bins(lams)
    w = np.zeros(len(lams))
    for i in range(len(lams)):
        a, b = max(lo[i], grid_lo), min(hi[i], grid[-1])
        if b > a:
            xs = np.concatenate(([a], grid[(grid > a) & (grid < b)], [b]))
            ys = np.interp(xs, grid, P)
            w[i] = np.trapezoid(ys, xs) / mult[i]
        if atom is not None and lo[i] <= atom[0] < hi[i]:
            w[i] += atom[1] / mult[i]
    return w


def weights_logpoisson(lams, Z, beta=2.0 / 3.0, C0=2.0):
    """Exact member masses for the log-Poisson exponents: K(t; Z) =
    (t - zeta_3t) Z = (2t/3 - C0 (1 - beta^t)) Z is the cumulant generating
    function of lambda = 2Z/3 + n ln(beta), n ~ Poisson(C0 Z)."""
    lo, hi, mult = lambda_bins(lams)
    mu = C0 * Z
    w = np.zeros(len(lams))
    logp = -mu
    for k in range(0, 400):
        if k > 0:
            logp += math.log(mu) - math.log(k)
        lam_k = 2.0 * Z / 3.0 + k * math.log(beta)
        for i in range(len(lams)):
            if lo[i] <= lam_k < hi[i]:
                w[i] += math.exp(logp) / mult[i]
    return w
