"""Pins of the oracle member solver (no GPU).

Each test fixes part of the solver with something other than the solver
itself: exact solutions (ABC/Beltrami decay), closed forms (Taylor-Green
initial dissipation rate), conservation laws (energy conservation of the
nonlinear term, the energy budget dE/dt = P - eps of Sec. II), convergence
orders of the time integrator, and the exact constant-power property of the
forcing (Sec. IV: injection rate fixed to exp(lambda) eps_bar).
"""
import math

import numpy as np
import pytest

import oracle as O


def grid(N):
    x = 2 * np.pi * np.arange(N) / N
    return np.meshgrid(x, x, x, indexing="ij")


def spectral(ufields):
    return np.ascontiguousarray(np.stack([O.rfft3(u) for u in ufields]))


def wavevectors(N):
    k = np.fft.fftfreq(N, 1.0 / N)
    kz = np.arange(N // 2 + 1)
    return np.meshgrid(k, k, kz, indexing="ij")


def full_sum(a, N):
    """Sum over the full spectrum of a quantity given on the half spectrum."""
    w = np.full(a.shape[-1], 2.0)
    w[0] = 1.0
    if N % 2 == 0:
        w[-1] = 1.0
    return float((a * w).sum())


def abc_field(N, A=1.0, B=0.7, C=0.4):
    X, Y, Zz = grid(N)
    return [A * np.sin(Zz) + C * np.cos(Y), B * np.sin(X) + A * np.cos(Zz), C * np.sin(Y) + B * np.cos(X)]


def test_dealias_cutoff_and_band_counts():
    assert [O.kc(N) for N in (32, 64, 128, 256, 384, 512)] == [10, 21, 42, 85, 127, 170]
    # brute-force count of |k| in [k_lo, k_hi] over the full spectrum
    for N, lo, hi in ((32, 1, 2), (64, 3, 5), (256, 6, 8)):
        k = np.fft.fftfreq(N, 1.0 / N)
        KX, KY, KZ = np.meshgrid(k, k, k, indexing="ij")
        k2 = KX ** 2 + KY ** 2 + KZ ** 2
        ref = int(np.count_nonzero((k2 >= lo * lo) & (k2 <= hi * hi)))
        assert O.band_modes(N, lo, hi) == ref
    assert O.band_modes(32, 1, 2) == 32


def test_white_noise_is_standard_normal():
    v = np.array([O.white_noise(7, i) for i in range(40000)])
    assert abs(v.mean()) < 0.02 and abs(v.std() - 1.0) < 0.02
    # known-answer check of the splitmix64 stream: first output for seed 0
    # (published test vector of splitmix64: 0xE220A8397B1DCDAF)
    h = 0xE220A8397B1DCDAF
    u1 = ((h >> 11) + 1) * 2.0 ** -53
    h2 = 0x6E789E6AA1B965F4
    u2 = ((h2 >> 11) + 1) * 2.0 ** -53
    ref = math.sqrt(-2 * math.log(u1)) * math.cos(2 * math.pi * u2)
    assert O.white_noise(0, 0) == pytest.approx(ref, rel=1e-15)


@pytest.mark.parametrize("N", [16, 24])
def test_abc_flow_nonlinear_term_vanishes(N):
    """ABC flow is Beltrami (omega = u), so u x omega = 0 and the projected
    nonlinear term is zero to rounding."""
    uh = spectral(abc_field(N))
    m = O.Member(N=N, nu=0.05, lam=-60.0, k_lo=1, k_hi=1.5)
    F, nl, umax, alpha = O.rhs(m, uh)
    assert np.abs(nl).max() < 1e-14
    assert umax == pytest.approx(math.sqrt(1.0) + 0.4, rel=0.3)


@pytest.mark.parametrize("rk", [2, 3])
def test_abc_flow_decays_exactly(rk):
    """With negligible injection (lambda = -60) the integrating factor makes
    the ABC decay exp(-nu k^2 t), k = 1, exact to rounding for any dt."""
    N, nu, dt, n = 16, 0.05, 0.3, 7
    uh = spectral(abc_field(N))
    m = O.Member(N=N, nu=nu, lam=-60.0, k_lo=1, k_hi=1.5, dt=dt, rk_order=rk)
    E0, _, _ = O.sums(m, uh)
    st, d = O.step(m, uh, n)
    assert st == 0
    assert d["E"] == pytest.approx(E0 * math.exp(-2 * nu * n * dt), rel=1e-12)
    assert d["t"] == pytest.approx(n * dt)


def test_taylor_green_initial_energy_rate():
    """Taylor-Green: dE/dt(0) = -6 nu E0 (all modes at |k|^2 = 3; the
    nonlinear term does no work)."""
    N, nu = 16, 0.03
    X, Y, Zz = grid(N)
    u = [np.sin(X) * np.cos(Y) * np.cos(Zz), -np.cos(X) * np.sin(Y) * np.cos(Zz), 0 * X]
    uh = spectral(u)
    m = O.Member(N=N, nu=nu, lam=-60.0, k_lo=1, k_hi=2)
    F, nl, _, _ = O.rhs(m, uh)
    KX, KY, KZ = wavevectors(N)
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    E0 = O.sums(m, uh)[0]
    assert E0 == pytest.approx(0.125, rel=1e-13)
    dEdt = full_sum(np.real(np.conj(uh) * (F - nu * k2 * uh)).sum(axis=0), N)
    assert dEdt == pytest.approx(-6 * nu * E0, rel=1e-12)
    # the nonlinear term of Taylor-Green is not zero, yet does no work
    assert np.abs(nl).max() > 1e-3
    assert abs(full_sum(np.real(np.conj(uh) * nl).sum(axis=0), N)) < 1e-14


def test_energy_budget_and_constant_power_forcing():
    """dE/dt = P - eps with P = exp(lambda) eps_bar exactly (Sec. II, the
    mean-injection argument; Sec. IV, constant-injection forcing)."""
    N = 16
    m = O.Member(N=N, nu=0.04, lam=0.7, k_lo=1, k_hi=2, seed=3)
    uh = O.initial_field(m)
    F, nl, umax, alpha = O.rhs(m, uh)
    KX, KY, KZ = wavevectors(N)
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    forcing = F - nl
    P = full_sum(np.real(np.conj(uh) * forcing).sum(axis=0), N)
    assert P == pytest.approx(math.exp(0.7) * 0.1, rel=1e-13)
    E, D, EB = O.sums(m, uh)
    assert alpha == pytest.approx(math.exp(0.7) * 0.1 / (2 * EB), rel=1e-14)
    D_ref = full_sum(m.nu * (k2 * np.abs(uh) ** 2).sum(axis=0), N)
    assert D == pytest.approx(D_ref, rel=1e-13)
    dEdt = full_sum(np.real(np.conj(uh) * (F - m.nu * k2 * uh)).sum(axis=0), N)
    assert dEdt == pytest.approx(P - D, rel=1e-12, abs=1e-14)
    # the forcing acts on the band only
    band = (k2 >= 1 - 1e-9) & (k2 <= 4 + 1e-9)
    assert np.abs(forcing[:, ~band]).max() == 0.0


def test_initial_field_properties():
    N = 24
    m = O.Member(N=N, nu=0.02, seed=11, init_energy=0.5)
    uh = O.initial_field(m)
    KX, KY, KZ = wavevectors(N)
    kc = O.kc(N)
    E = O.sums(m, uh)[0]
    assert E == pytest.approx(0.5, rel=1e-13)
    div = KX * uh[0] + KY * uh[1] + KZ * uh[2]
    assert np.abs(div).max() < 1e-15
    outside = (np.abs(KX) > kc) | (np.abs(KY) > kc) | (KZ > kc)
    assert np.abs(uh[:, outside]).max() == 0.0
    # shell spectrum follows s^4 exp(-s^2/2)
    s = np.rint(np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)).astype(int)
    w = np.where(KZ == 0, 1.0, 2.0)
    Es = np.bincount(s.ravel(), weights=(0.5 * w * (np.abs(uh) ** 2).sum(axis=0)).ravel())
    target = np.array([si ** 4 * math.exp(-0.5 * si * si) for si in range(len(Es))])
    occ = Es > 0
    ratio = Es[occ] / target[occ]
    assert np.allclose(ratio, ratio[0], rtol=1e-12)
    # deterministic in the seed, different across seeds
    assert np.array_equal(uh, O.initial_field(m))
    m2 = O.Member(N=N, nu=0.02, seed=12)
    assert np.abs(O.initial_field(m2) - uh).max() > 1e-3


def _run(m, uh0, dt, T):
    uh = uh0.copy()
    mm = O.Member(**{**m.__dict__, "dt": dt})
    st, d = O.step(mm, uh, int(round(T / dt)))
    assert st == 0
    return uh


@pytest.mark.parametrize("rk,order", [(2, 2), (3, 3)])
def test_time_integrator_convergence_order(rk, order):
    """Self-convergence under dt halving: error ratios 2^p."""
    N, T = 12, 0.4
    m = O.Member(N=N, nu=0.05, lam=0.5, k_lo=1, k_hi=2, seed=5, rk_order=rk, init_energy=1.0)
    uh0 = O.initial_field(m)
    ref = _run(m, uh0, T / 64, T)
    errs = [np.linalg.norm(_run(m, uh0, T / n, T) - ref) for n in (4, 8, 16)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - order) < 0.35 for r in rates), (errs, rates)


def test_solenoidal_after_steps_and_cfl_step():
    N = 16
    m = O.Member(N=N, nu=0.03, lam=1.0, k_lo=1, k_hi=2, seed=2, dt=-1.0, cfl=0.2, rk_order=3)
    uh = O.initial_field(m)
    _, _, umax, _ = O.rhs(m, uh)
    st, d = O.step(m, uh, 1)
    assert st == 0
    assert d["dt"] == pytest.approx(0.2 * (2 * math.pi / N) / umax, rel=1e-14)
    KX, KY, KZ = wavevectors(N)
    div = KX * uh[0] + KY * uh[1] + KZ * uh[2]
    assert np.abs(div).max() < 1e-14 * np.abs(uh).max() * N
    # cap on the adaptive step
    m2 = O.Member(**{**m.__dict__, "dt_max": 1e-4})
    st, d2 = O.step(m2, O.initial_field(m2), 1)
    assert d2["dt"] == 1e-4
