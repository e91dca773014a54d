"""Statistics in Kolmogorov units: runs at different viscosity compared on
common axes.

The paper compares the ensemble's predictions with reference simulations
at other Reynolds numbers in Kolmogorov-normalised units (Sec. V and VI:
gradients in units of <Tr S^2>, dissipation in units of its mean); a single
reference run at another viscosity than the members' is compared the same
way.  The library's histogram axes are set by eps_norm and nu_norm
(q0 = eps_norm / (2 nu_norm) = <Tr S^2>, the dissipation axis eps/eps_norm,
the enstrophy axis omega^2 nu_norm / eps_norm), so a run binned with its
own eps and nu lands on Kolmogorov-normalised axes.

Exact check from the scaling symmetry of the Navier-Stokes equations: with
u -> a u, nu -> a nu, eps -> a^3 eps and t -> t / a the discrete
trajectory maps onto itself (CFL step dt -> dt / a, forcing amplitude
alpha -> a alpha).  With a = 2 every rescaling is by a power of two, exact
in binary floating point, so the two runs agree to the last bit up to the
powers of two, and their histograms in their own Kolmogorov units are equal
count for count.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("N,k_lo,k_hi", [(32, 1, 2), (64, 3, 5)])
def test_rescaled_runs_agree_in_kolmogorov_units(E, N, k_lo, k_hi):
    a = 2.0
    nu, eps, e0 = 0.02, 0.1, 0.5
    kw = dict(N=N, lam=0.3, k_lo=k_lo, k_hi=k_hi, dt=-1, cfl=0.2, rk_order=3, seed=11)
    m1 = E.Member(nu=nu, eps_bar=eps, init_energy=e0, **kw)
    m2 = E.Member(nu=a * nu, eps_bar=a ** 3 * eps, init_energy=a * a * e0, **kw)
    hk = dict(qr_bins=64, q_lim=10.0, r_lim=10.0, tail_bins=128, tail_lo=-6.0, tail_hi=6.0, grad_bins=64,
              grad_lim=8.0)
    e1 = E.Ensemble([m1], hist=E.hist_spec(eps_norm=eps, nu_norm=nu, **hk))
    e2 = E.Ensemble([m2], hist=E.hist_spec(eps_norm=a ** 3 * eps, nu_norm=a * nu, **hk))
    for e in (e1, e2):
        e.step(10)
        for s in range(4):
            e.step(5)
            e.gradient_stats(accumulate=s > 0)
    d1, d2 = e1.diagnostics()[0], e2.diagnostics()[0]
    assert d2["dt"] == d1["dt"] / a
    assert d2["t"] == d1["t"] / a
    assert d2["E"] == a * a * d1["E"]
    assert d2["diss"] == a ** 3 * d1["diss"]
    assert np.array_equal(e2.field(0), a * e1.field(0))
    c1, mom1 = e1.stats()
    c2, mom2 = e2.stats()
    assert c1[0, -2 - (2 * 64 + 4)] == 4 * N ** 3          # npoints (counters before the gradient block)
    assert np.array_equal(c1, c2)
    # the mixtures (one member, weight 1) in Kolmogorov units are the same PDFs
    p1 = e1.mixture(kind=E.W_USER, user=[1.0], renormalize=False)
    p2 = e2.mixture(kind=E.W_USER, user=[1.0], renormalize=False)
    for k in ("pdf_qr", "pdf_eps", "pdf_ens", "pdf_long", "pdf_trans"):
        assert np.array_equal(p1[k], p2[k]), k
    for k in p1["ratios"]:
        assert p1["ratios"][k] == pytest.approx(p2["ratios"][k], rel=1e-12)
    e1.close()
    e2.close()
