"""Pins of the oracle lambda weights and mixture (no GPU).

Pins: the mean-injection constraint int P e^lambda = 1 (Sec. II), the
convolution property P(.; 2Z) = P(.; Z) * P(.; Z) (Sec. III), the printed
bin mass 3.1e-6 of the member at lambda = 3.93 for R_lambda = 1300 with
ens256 (Sec. VII), the printed cost ratio 7.8e4 (Sec. VI), Z = 0 giving the
central member (Sec. VII), the truncated Gaussian of the Appendix, and the
numerical inverse Laplace transform (Sec. VII) reproducing the Gaussian
and, for saturating exponents, the exact compound-Poisson law below.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import oracle.mixture as M

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_gaussian_pdf_moments_and_constraint():
    c, Z = 0.023, 2.0
    lam = np.linspace(-30, 30, 600001)
    P = M.gauss_pdf(lam, c, Z)
    assert np.trapezoid(P, lam) == pytest.approx(1.0, abs=1e-12)
    assert np.trapezoid(P * np.exp(lam), lam) == pytest.approx(1.0, abs=1e-10)
    mu, s = M.gauss_params(c, Z)
    assert np.trapezoid(P * lam, lam) == pytest.approx(mu, abs=1e-12)
    assert np.trapezoid(P * (lam - mu) ** 2, lam) == pytest.approx(s * s, rel=1e-10)
    # K(t; Z) = log int P e^{lambda t} equals 9c(t^2 - t)Z/2 and (t - zeta_3t) Z
    for t in (0.5, 1.0, 2.0, 3.0):
        K = math.log(np.trapezoid(P * np.exp(lam * t), lam))
        assert K == pytest.approx(9 * c * (t * t - t) * Z / 2, abs=1e-9)
        assert K == pytest.approx(M.K_from_zeta(t, Z, lambda p: M.zeta_quadratic(p, c)), abs=1e-9)


def test_convolution_property():
    c, Z = 0.023, 1.3
    lam = np.linspace(-20, 20, 8001)
    dl = lam[1] - lam[0]
    P1 = M.gauss_pdf(lam, c, Z)
    conv = np.convolve(P1, P1, mode="same") * dl
    P2 = M.gauss_pdf(lam, c, 2 * Z)
    assert np.abs(conv - P2).max() < 1e-9 * P2.max()


def test_paper_bin_mass_pin():
    g = golden()["bin_mass_lambda_3.93"]
    lams = np.linspace(g["lambda_min"], g["lambda_max"], g["n_members"])
    Z = M.Z_from_Rlambda(g["R_ref"], g["R_ens"])
    w, covered = M.member_weights(lams, "gauss_paper", c=g["c"], Z=Z, renormalize=False)
    i = int(np.argmin(np.abs(lams - g["lambda"])))
    assert abs(lams[i] - g["lambda"]) < 0.02
    # the paper prints 3.1e-6 (two digits)
    assert round(w[i] * 1e7) / 10 == pytest.approx(g["mass"] * 1e6, abs=0.051)
    assert 0.999 < covered <= 1.0


def test_paper_cost_ratio_pin():
    g = golden()["cost_ratio"]
    r = M.cost_ratio(g["R_ref"], g["R_ens"], g["n"])
    assert r == pytest.approx(g["value"], rel=0.01)


def test_scale_gap_zero_gives_central_member():
    lams = np.linspace(-3, 3, 7)
    w, covered = M.member_weights(lams, "gauss_paper", c=0.023, Z=0.0)
    assert w[3] == 1.0 and w.sum() == 1.0


def test_weights_bins_and_duplicates():
    lams = np.array([0.0, 1.0, 1.0, 3.0])
    lo, hi, mult = M.lambda_bins(lams)
    assert list(lo) == [-0.5, 0.5, 0.5, 2.0] and list(hi) == [0.5, 2.0, 2.0, 4.0]
    assert list(mult) == [1, 2, 2, 1]
    w, cov = M.member_weights(lams, "gauss", mu=0.5, sigma=1.0, renormalize=False)
    ref_mid = (M._norm_cdf(1.5) - M._norm_cdf(0.0)) / 2
    assert w[1] == pytest.approx(ref_mid, rel=1e-14) and w[1] == w[2]
    assert cov == pytest.approx(M._norm_cdf(3.5) - M._norm_cdf(-1.0), rel=1e-14)
    wn, _ = M.member_weights(lams, "gauss", mu=0.5, sigma=1.0)
    assert wn.sum() == pytest.approx(1.0, abs=1e-15)
    # a single member owns the whole line
    w1, c1 = M.member_weights([0.4], "gauss", mu=-3, sigma=0.1, renormalize=False)
    assert w1[0] == 1.0 and c1 == 1.0


def test_truncated_gaussian():
    c, Z = 0.023, 2.0
    mu, s, cut = M.truncated_gauss_params(c, Z)
    assert cut == Z
    lam = np.linspace(-30, Z, 800001)
    P = np.exp(-(lam - mu) ** 2 / (18 * c * Z))
    P /= np.trapezoid(P, lam)
    assert np.trapezoid(P * np.exp(lam), lam) == pytest.approx(1.0, abs=1e-8)
    # bin masses: nothing above the cut
    lams = np.linspace(-3, 4, 15)
    w, cov = M.member_weights(lams, "trunc_gauss", c=c, Z=Z, renormalize=False)
    assert np.all(w[lams - 0.25 >= Z] == 0.0)
    assert 0.99 < cov <= 1.0 + 1e-12


def test_inverse_laplace_reproduces_gaussian():
    c, Z = 0.023, 2.5
    lam = np.linspace(-12, 12, 1024, endpoint=False)
    P = M.lambda_pdf_from_K(lambda t: 9 * c * (t * t - t) * Z / 2, lam)
    assert np.abs(P - M.gauss_pdf(lam, c, Z)).max() < 1e-10


def test_mixture_of_counts():
    h = O.HistSpec(qr_bins=4, tail_bins=4, q_lim=2.0, r_lim=2.0, tail_lo=-1.0, tail_hi=1.0)
    L = h.counts_len
    rng = np.random.default_rng(0)
    counts = rng.integers(0, 100, size=(3, L)).astype(np.uint64)
    npts = counts[:, :16].sum(axis=1) + counts[:, 16 + 8]   # in range + qr_out
    counts[:, 16 + 8 + 6] = npts
    w = np.array([0.2, 0.5, 0.3])
    qr, e, ww = M.mix_counts(counts, w, h)
    # integrals of the mixed PDFs equal the mixed in-range fractions
    frac = (w * counts[:, :16].sum(axis=1) / npts).sum()
    assert (qr * (1.0 * 1.0)).sum() == pytest.approx(frac, rel=1e-14)
    # a single member with weight 1 reproduces its normalised histogram
    qr1, _, _ = M.mix_counts(counts[1:2], np.array([1.0]), h)
    assert np.allclose(qr1.ravel(), counts[1, :16] / npts[1], rtol=1e-15)


def test_gradient_pdf_mixture():
    """Mixed gradient-component PDFs integrate to the mixed in-range
    fractions (3 and 6 samples per point), and one member with weight 1
    gives its own normalised histogram."""
    h = O.HistSpec(qr_bins=2, tail_bins=2, grad_bins=5, grad_lim=2.5)
    L = h.counts_len
    off = 4 + 4
    rng = np.random.default_rng(1)
    counts = np.zeros((3, L), dtype=np.uint64)
    npts = np.array([1000, 2000, 1500])
    for i in range(3):
        counts[i, off + 6] = npts[i]
        counts[i, off + 8: off + 13] = rng.multinomial(3 * npts[i] - 7, np.ones(5) / 5)
        counts[i, off + 13: off + 18] = rng.multinomial(6 * npts[i] - 11, np.ones(5) / 5)
    w = np.array([0.2, 0.5, 0.3])
    lon, tra = M.mix_gradient_pdfs(counts, w, h)
    db = 1.0
    frac_l = (w * counts[:, off + 8: off + 13].sum(axis=1) / (3 * npts)).sum()
    frac_t = (w * counts[:, off + 13: off + 18].sum(axis=1) / (6 * npts)).sum()
    assert lon.sum() * db == pytest.approx(frac_l, rel=1e-14)
    assert tra.sum() * db == pytest.approx(frac_t, rel=1e-14)
    l1, _ = M.mix_gradient_pdfs(counts[1:2], np.array([1.0]), h)
    assert np.allclose(l1, counts[1, off + 8: off + 13] / (3.0 * npts[1]), rtol=1e-15)


def test_moment_ratios_of_gaussian_components():
    """Gaussian gradient components: S = 0, F = 3, H = 15."""
    mixed = np.zeros(48)
    for comp in range(9):
        s2 = 1.0 + comp
        mixed[4 * comp + 0] = s2
        mixed[4 * comp + 1] = 0.0
        mixed[4 * comp + 2] = 3 * s2 ** 2
        mixed[4 * comp + 3] = 15 * s2 ** 3
    r = M.gradient_moment_ratios(mixed)
    assert r["S_long"] == 0.0
    # per-component averages of moments of different variances: F of the average
    assert r["F_long"] == pytest.approx(3 * np.mean([1, 25, 81]) / np.mean([1, 5, 9]) ** 2)


def test_hellinger():
    p = np.array([0.5, 0.5, 0.0])
    assert M.hellinger(p, p) == 0.0
    assert M.hellinger(p, np.array([0.0, 0.0, 1.0])) == pytest.approx(1.0)


def test_scale_gap_fit():
    """Members on R_lambda = R0 exp(lambda/6) recover R0; the paper's
    R_ens = 63, R_ref = 1300 give Z = 1.5 ln(1300/63)."""
    lams = np.linspace(-3, 3, 13)
    R = 63.0 * np.exp(lams / 6.0)
    assert M.fit_R0(lams, R) == pytest.approx(63.0, rel=1e-12)
    assert M.scale_gap(lams, R, 1300.0) == pytest.approx(1.5 * math.log(1300 / 63), rel=1e-12)
    # only lambda >= 0 enters the fit
    R2 = R.copy()
    R2[lams < 0] *= 5.0
    assert M.fit_R0(lams, R2) == pytest.approx(63.0, rel=1e-12)


def test_nelkin_exponents_closed_forms():
    """K41 (c = 0): rho_m = m/2; quadratic zeta: rho solves a quadratic."""
    k41 = lambda p: p / 3.0
    for m in (2, 3, 4, 6):
        assert M.nelkin_rho(m, k41) == pytest.approx(m / 2.0, abs=1e-12)
    c = 0.023
    z = lambda p: M.zeta_quadratic(p, c)
    for m in (2, 3, 4, 6):
        # rho = m - (m+rho)/3 + c((m+rho)^2 - 3(m+rho))/2  ->  a rho^2 + b rho + d = 0
        a = c / 2.0
        b = -(1 + 1 / 3.0) + c * (2 * m - 3) / 2.0
        d = m - m / 3.0 + c * (m * m - 3 * m) / 2.0
        disc = math.sqrt(b * b - 4 * a * d)
        roots = [(-b - disc) / (2 * a), (-b + disc) / (2 * a)]
        ref = min(roots, key=lambda r: abs(r - m / 2.0))
        assert M.nelkin_rho(m, z) == pytest.approx(ref, abs=1e-10)
    S, F, H = M.ratio_exponents(z)
    assert S < 0.2 and F > 0 and H > F   # intermittency grows with order


def test_numeric_weights_reproduce_gaussian_and_logpoisson_constraint():
    c, Z = 0.023, 2.0
    lams = np.linspace(-3, 2, 11)
    Kq = lambda t, Zz: 9 * c * (t * t - t) * Zz / 2
    wn = M.weights_numeric(lams, Kq, Z)
    wg, _ = M.member_weights(lams, "gauss_paper", c=c, Z=Z, renormalize=False)
    # trapezoid rule on the 60/65536 grid: error <= h^2 max|P''| (bin width)/12 ~ 7e-8
    assert np.abs(wn - wg).max() < 2e-7
    # log-Poisson: exact masses; K(1; Z) = 0 is the mean-injection constraint
    beta, C0 = 2.0 / 3.0, 2.0
    assert M.zeta_logpoisson(3.0, beta, C0) == pytest.approx(1.0, abs=1e-15)
    mu = C0 * Z
    s = sum(math.exp(-mu + k * math.log(mu) - math.lgamma(k + 1)) * math.exp(2 * Z / 3 + k * math.log(beta))
            for k in range(200))
    assert s == pytest.approx(1.0, abs=1e-12)
    lams = np.linspace(-4.0, 1.5, 23)
    w = M.weights_logpoisson(lams, Z)
    assert 0.99 < w.sum() <= 1.0 + 1e-12


def _rational_exact(lams, Z, beta):
    """Exact bin masses for zeta_p = (1+3b)p/(3(1+bp)).  K(t; Z) = Z t +
    A Z (1/(1 + 3 b t) - 1), A = (1+3b)/(3b), is the cumulant generating
    function of lambda = Z - 3 b G, G ~ Gamma(N, 1), N ~ Poisson(A Z) (G = 0
    for N = 0): a closed form independent of any transform."""
    from scipy.special import gammainc
    A = (1 + 3 * beta) / (3 * beta)
    mu = A * Z
    lo, hi, mult = M.lambda_bins(lams)
    w = np.zeros(len(lams))
    for i in range(len(lams)):
        g_hi = (Z - lo[i]) / (3 * beta)       # lambda >= lo  <=>  G <= g_hi
        g_lo = (Z - hi[i]) / (3 * beta)
        s = math.exp(-mu) if lo[i] <= Z < hi[i] else 0.0
        for N in range(1, int(mu + 40 * math.sqrt(mu) + 60)):
            pN = math.exp(-mu + N * math.log(mu) - math.lgamma(N + 1))
            F = lambda g: gammainc(N, g) if g > 0 else 0.0
            s += pN * (F(g_hi) - F(g_lo))
        w[i] = s / mult[i]
    return w


@pytest.mark.parametrize("Z", [0.5, 2.0, 4.5])
def test_rational_numeric_inversion_matches_compound_poisson(Z):
    beta = 0.05
    A = (1 + 3 * beta) / (3 * beta)
    zeta = lambda p: M.zeta_rational(p, beta)
    assert zeta(3.0) == pytest.approx(1.0, abs=1e-15)
    assert zeta(1e12) == pytest.approx(A, rel=1e-10)
    lams = np.linspace(-3, 3, 64)
    atom = M.saturation_atom(A, Z)
    w = M.weights_numeric(lams, lambda t, Zz: (t - zeta(3 * t)) * Zz, Z, atom=atom)
    ref = _rational_exact(lams, Z, beta)
    # the continuous part jumps by J = e^{-AZ} A Z / (3 beta) at lambda = Z;
    # its Gibbs residual in a bin mass stays below 2e-3 J dl
    dl = 60.0 / 65536
    J = math.exp(-A * Z) * A * Z / (3 * beta)
    assert np.abs(w - ref).max() < max(2e-3 * J * dl, 1e-8)
    # saturation: no mass above lambda_max = Z (Appendix)
    grid = np.linspace(-30, 30, 65536, endpoint=False)
    P = M.lambda_pdf_from_K(lambda t: (t - zeta(3 * t)) * Z, grid, atom)
    assert abs(P[grid > Z + 0.05].sum() * dl) < max(2e-3 * J * dl, 1e-12)


def _power_law_members(lams, rho, c):
    """Member moments of an exactly scaling ensemble (Sec. III, Eq.
    scaling_equation_2 at fixed nu and L): <A^m>_lambda ~ exp(lambda (m +
    rho_m) / 3), negative for m = 3 (negative skewness); all nine components
    alike.  Layout of the 48 moment sums with one point per member."""
    mom = np.zeros((len(lams), 48))
    for j, m in enumerate((2, 3, 4, 6)):
        v = np.exp(np.asarray(lams) * (m + rho[m]) / 3.0) * (-1.0 if m == 3 else 1.0)
        for comp in range(9):
            mom[:, 4 * comp + j] = v
    return mom


def test_mixture_ratios_follow_nelkin_exponents():
    """Mixing exactly scaling members with P(lambda; Z) gives skewness,
    flatness and hyper-flatness that scale with R_lambda ~ exp(2Z/3) as the
    Nelkin relation predicts (Sec. III, Eq. nelkin_rhom; Sec. VII):
    d ln|S| / d ln R = 2 rho3 - 3 rho2, d ln F / d ln R = 2 rho4 - 4 rho2,
    d ln H / d ln R = 2 rho6 - 6 rho2."""
    c = 0.023
    zeta = lambda p: M.zeta_quadratic(p, c)
    rho = {m: M.nelkin_rho(m, zeta) for m in (2, 3, 4, 6)}
    lams = np.linspace(-9.0, 12.0, 2048)
    mom = _power_law_members(lams, rho, c)
    npts = np.ones(len(lams))
    out = {}
    for Z in (1.0, 3.0):
        w, _ = M.member_weights(lams, "gauss_paper", c=c, Z=Z, renormalize=False)
        out[Z] = M.gradient_moment_ratios(M.mix_moments(mom, npts, w))
    dlnR = 2.0 / 3.0 * (3.0 - 1.0)
    slope = lambda k: (math.log(abs(out[3.0][k])) - math.log(abs(out[1.0][k]))) / dlnR
    S, F, H = M.ratio_exponents(zeta)
    assert slope("S_long") == pytest.approx(S, abs=2e-3)
    assert slope("F_long") == pytest.approx(F, abs=2e-3)
    assert slope("H_long") == pytest.approx(H, abs=2e-3)
    assert slope("F_trans") == pytest.approx(F, abs=2e-3)
