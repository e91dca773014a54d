"""Scaling-exponent theory through the C ABI against the FP64 oracle:
lambda PDFs and member weights of the quadratic, rational (saturating) and
log-Poisson zeta_p families (Sec. III; Sec. VII numerical inverse Laplace
transform; Appendix saturation), Nelkin exponents (Sec. III), the
scale-gap fit (Sec. V), and a mixture driven by log-Poisson weights.

Tolerances: the device evaluates the same FP64 sums as the oracle, in a
different order (a radix-2 Stockham FFT against numpy's FFT), so the grid
densities agree to 1e-12 absolute (values O(1), 16 butterfly stages); bin masses
to 1e-12; bisection roots and the closed-form fit to 1e-12.
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.mixture as OM

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2506_23712_gb300 import build as B
    B.build()
    import paper_2506_23712_gb300.ens as ens
    return ens


C = 0.023
BETA = 0.05
A_RAT = (1 + 3 * BETA) / (3 * BETA)     # zeta_inf of the rational family


def K_of(zeta):
    return lambda t, Z: (t - zeta(3.0 * t)) * Z


def zq(p):
    return OM.zeta_quadratic(p, C)


def zr(p):
    return OM.zeta_rational(p, BETA)


def oracle_grid():
    return np.linspace(-30.0, 30.0, 65536, endpoint=False)


def test_grid_matches_oracle(E):
    assert np.array_equal(E.lambda_grid(), oracle_grid())


@pytest.mark.parametrize("Z", [0.5, 2.0, 4.5])
def test_lambda_pdf_quadratic_and_rational(E, Z):
    grid = oracle_grid()
    ref = OM.lambda_pdf_from_K(lambda t: K_of(zq)(t, Z), grid)
    got = E.ens_lambda_pdf(E.zeta_spec("quadratic", c=C), Z)
    assert np.abs(got - ref).max() < 1e-12
    # and the closed-form Gaussian of Sec. IV within the grid's aliasing error
    assert np.abs(got - OM.gauss_pdf(grid, C, Z)).max() < 1e-10
    atom = OM.saturation_atom(A_RAT, Z)
    ref_r = OM.lambda_pdf_from_K(lambda t: K_of(zr)(t, Z), grid, atom)
    got_r = E.ens_lambda_pdf(E.zeta_spec("rational", beta=BETA), Z)
    assert np.abs(got_r - ref_r).max() < 1e-12


@pytest.mark.parametrize("n,Z", [(64, 2.0), (13, 0.7), (257, 3.5)])
def test_lambda_weights_match_oracle(E, n, Z):
    lams = np.linspace(-3.0, 3.0, n)
    lams[n // 3] = lams[n // 3 + 1]                 # a shared lambda value
    w, cov = E.ens_lambda_weights(E.zeta_spec("quadratic", c=C), Z, lams)
    ref = OM.weights_numeric(lams, K_of(zq), Z)
    assert np.abs(w - ref).max() < 1e-12
    assert cov == pytest.approx(ref.sum(), abs=1e-12)
    # the quadratic family against the closed-form Gaussian bin masses
    wg, _ = OM.member_weights(lams, "gauss_paper", c=C, Z=Z, renormalize=False)
    assert np.abs(w - wg).max() < 2e-7
    # the rational family, point mass at lambda = Z included
    w, cov = E.ens_lambda_weights(E.zeta_spec("rational", beta=BETA), Z, lams)
    ref = OM.weights_numeric(lams, K_of(zr), Z, atom=OM.saturation_atom(A_RAT, Z))
    assert np.abs(w - ref).max() < 1e-12
    assert 0.9 < cov <= 1.0 + 1e-9


@pytest.mark.parametrize("beta,C0,Z", [(2.0 / 3.0, 2.0, 2.0), (0.6, 1.5, 1.0)])
def test_logpoisson_weights_exact(E, beta, C0, Z):
    lams = np.linspace(-4.0, 1.5, 23)
    w, cov = E.ens_lambda_weights(E.zeta_spec("logpoisson", beta=beta, C0=C0), Z, lams)
    ref = OM.weights_logpoisson(lams, Z, beta=beta, C0=C0)
    assert np.allclose(w, ref, rtol=1e-13, atol=1e-300)
    assert cov == pytest.approx(ref.sum(), rel=1e-13)


def test_nelkin_and_ratio_exponents(E):
    m = np.array([2.0, 3.0, 4.0, 6.0])
    for spec, zeta in ((E.zeta_spec("quadratic", c=C), lambda p: OM.zeta_quadratic(p, C)),
                       (E.zeta_spec("logpoisson"), OM.zeta_logpoisson),
                       (E.zeta_spec("rational", beta=BETA), zr)):
        rho = E.ens_nelkin_exponents(spec, m)
        ref = [OM.nelkin_rho(mm, zeta) for mm in m]
        assert np.allclose(rho, ref, rtol=0, atol=1e-12)
        assert np.allclose(E.ens_ratio_exponents(spec), OM.ratio_exponents(zeta), rtol=0, atol=1e-12)
    # K41 (c = 0): rho_m = m/2 exactly, no intermittency corrections
    rho = E.ens_nelkin_exponents(E.zeta_spec("quadratic", c=0.0), m)
    assert np.allclose(rho, m / 2, atol=1e-12)


def test_scale_gap(E):
    rng = np.random.default_rng(3)
    lams = np.linspace(-3, 3, 17)
    R = 63.0 * np.exp(lams / 6.0) * np.exp(0.05 * rng.standard_normal(lams.size))
    Z, R0 = E.ens_scale_gap(lams, R, 1300.0)
    assert R0 == pytest.approx(OM.fit_R0(lams, R), rel=1e-12)
    assert Z == pytest.approx(OM.scale_gap(lams, R, 1300.0), rel=1e-12)


def test_invalid_arguments_rejected(E):
    with pytest.raises(E.EnsError):
        E.ens_lambda_weights(E.zeta_spec("logpoisson", beta=1.5), 1.0, [0.0, 1.0])
    with pytest.raises(E.EnsError):
        E.ens_lambda_weights(E.zeta_spec("quadratic"), 0.0, [0.0, 1.0])
    with pytest.raises(E.EnsError):
        E.ens_lambda_weights(E.zeta_spec("quadratic"), 1.0, [0.0, math.nan])
    with pytest.raises(E.EnsError):
        E.ens_lambda_pdf(E.zeta_spec("logpoisson"), 1.0)
    with pytest.raises(E.EnsError):
        E.ens_scale_gap([-1.0, -2.0], [50.0, 40.0], 1300.0)     # no member with lambda >= 0


def test_logpoisson_weights_drive_mixture(E):
    """User weights from the log-Poisson law through ens_mixture_host equal
    the oracle mixture of the same counts (Sec. II, Eq. pdf_superposition)."""
    import ens_inputs as I
    lams = np.linspace(-3.0, 1.5, 10)
    h = E.hist_spec(qr_bins=8, tail_bins=16)
    oh = O.HistSpec(qr_bins=8, tail_bins=16)
    counts = I.synthetic_member_counts(list(lams), 8, 16, 20000, seed=5)
    mom = np.random.default_rng(5).standard_normal((lams.size, 48)) ** 2
    w, _ = E.ens_lambda_weights(E.zeta_spec("logpoisson"), 2.0, lams)
    got = E.ens_mixture_host(lams, counts, mom, h, kind=E.W_USER, user=w, renormalize=False)
    qr, pe, pw = OM.mix_counts(counts, w, oh)
    assert np.allclose(got["pdf_qr"], qr, rtol=1e-12, atol=1e-15)
    assert np.allclose(got["pdf_eps"], pe, rtol=1e-12, atol=1e-15)
    assert np.allclose(got["pdf_ens"], pw, rtol=1e-12, atol=1e-15)
