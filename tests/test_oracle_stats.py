"""Pins of the oracle gradient statistics (no GPU).

Q = -1/2 Tr A^2, R = -1/3 Tr A^3 (Sec. V), eps = 2 nu Tr S^2 and omega^2
(Sec. VI).  Pins: closed forms for constant tensors, the periodic-box
identities <Q> = <R> = 0 and <eps> = nu <omega^2> (exact on the grid for
dealiased fields, whose pair and triple products do not alias onto k = 0),
tr A = 0, agreement of <eps> with the spectral dissipation, and histogram
counts against an independent brute-force binning.
"""
import math

import numpy as np
import pytest

import ens_inputs as I
import oracle as O


def const_A(a, N=4):
    A = np.empty((3, 3, N, N, N))
    for i in range(3):
        for j in range(3):
            A[i, j] = a[i][j]
    return A


def test_invariants_closed_forms():
    # pure rotation about z with angular rate a: omega_z = 2a, Q = omega^2/4, R = 0
    a = 0.7
    Q, R, eps, ens = O.invariants(const_A([[0, -a, 0], [a, 0, 0], [0, 0, 0]]), nu=0.1)
    assert np.allclose(Q, a * a, rtol=1e-15) and np.allclose(R, 0.0, atol=1e-16)
    assert np.allclose(ens, 4 * a * a, rtol=1e-15) and np.allclose(eps, 0.0, atol=1e-16)
    # pure strain diag(a, b, -a-b): Q = -(a^2+ab+b^2), R = ab(a+b), eps = 2 nu S:S
    a, b, nu = 0.3, -1.1, 0.02
    Q, R, eps, ens = O.invariants(const_A([[a, 0, 0], [0, b, 0], [0, 0, -a - b]]), nu=nu)
    assert np.allclose(Q, -(a * a + a * b + b * b), rtol=1e-14)
    assert np.allclose(R, a * b * (a + b), rtol=1e-14)
    assert np.allclose(eps, 2 * nu * (a * a + b * b + (a + b) ** 2), rtol=1e-14)
    assert np.allclose(ens, 0.0, atol=1e-16)
    # a generic traceless tensor: Cayley-Hamilton gives R = -det A and Q = sum
    # of the principal 2x2 minors (pairwise products of eigenvalues)
    rng = np.random.default_rng(1)
    M = rng.standard_normal((3, 3))
    M -= np.trace(M) / 3 * np.eye(3)
    Q, R, _, _ = O.invariants(const_A(M.tolist()), nu=1.0)
    assert R[0, 0, 0] == pytest.approx(-np.linalg.det(M), rel=1e-12)
    eig = np.linalg.eigvals(M)
    assert Q[0, 0, 0] == pytest.approx(np.real(eig[0] * eig[1] + eig[1] * eig[2] + eig[0] * eig[2]), rel=1e-12)


def test_gradient_of_single_mode():
    """A_ij = d_j u_i of u = (0, sin(2x + z), 0): A_21 = 2 cos, A_23 = cos."""
    N = 8
    x = 2 * np.pi * np.arange(N) / N
    X, Y, Zz = np.meshgrid(x, x, x, indexing="ij")
    u = [0 * X, np.sin(2 * X + Zz), 0 * X]
    uh = np.stack([O.rfft3(f) for f in u])
    A = O.gradient(uh)
    ref = np.zeros_like(A)
    ref[1, 0] = 2 * np.cos(2 * X + Zz)
    ref[1, 2] = np.cos(2 * X + Zz)
    assert np.abs(A - ref).max() < 1e-13


@pytest.mark.parametrize("N", [16, 24])
def test_periodic_box_identities(N):
    m = O.Member(N=N, nu=0.03, seed=N)
    uh = O.initial_field(m)
    A = O.gradient(uh)
    Q, R, eps, ens = O.invariants(A, m.nu)
    assert abs(Q.mean()) < 1e-13 * np.abs(Q).mean()
    assert abs(R.mean()) < 1e-13 * np.abs(R).mean()
    assert eps.mean() == pytest.approx(m.nu * ens.mean(), rel=1e-12)
    assert np.abs(A[0, 0] + A[1, 1] + A[2, 2]).max() < 1e-13 * np.abs(A).max()
    # <eps> equals the spectral dissipation nu sum k^2 |uh|^2
    assert eps.mean() == pytest.approx(O.sums(m, uh)[1], rel=1e-12)


def brute_bins(x, edges):
    """Independent binning: count of float32 edges <= float32(x), minus one."""
    xf = np.float32(x)
    return np.searchsorted(edges, xf, side="right") - 1


def test_histograms_against_brute_force():
    N = 8
    m = O.Member(N=N, nu=0.05, seed=4, init_energy=3.0)
    uh = O.initial_field(m)
    h = O.HistSpec(qr_bins=16, q_lim=4.0, r_lim=4.0, tail_bins=32, tail_lo=-3.0, tail_hi=2.0,
                   eps_norm=0.1, nu_norm=0.05)
    counts, mom = O.gradient_stats(uh, m.nu, h)
    qr, he, hw, ctr = O.split_counts(counts, h)
    A = O.gradient(uh)
    Q, R, eps, ens = O.invariants(A, m.nu)
    q0 = h.eps_norm / (2 * h.nu_norm)
    eq = np.array([np.float32(-4.0 + 8.0 * b / 16) for b in range(17)], dtype=np.float32)
    et = np.array([np.float32(10.0 ** (-3.0 + 5.0 * b / 32)) for b in range(33)], dtype=np.float32)
    bq = brute_bins((Q / q0).ravel(), eq)
    br = brute_bins((R / q0 ** 1.5).ravel(), eq)
    ok = (bq >= 0) & (bq < 16) & (br >= 0) & (br < 16)
    ref = np.zeros((16, 16), dtype=np.int64)
    np.add.at(ref, (bq[ok], br[ok]), 1)
    assert np.array_equal(qr.astype(np.int64), ref)
    assert ctr[0] == np.count_nonzero(~ok)
    for vals, hist, cu, co in ((eps / h.eps_norm, he, ctr[1], ctr[2]),
                               (ens * h.nu_norm / h.eps_norm, hw, ctr[3], ctr[4])):
        b = brute_bins(vals.ravel(), et)
        inr = (b >= 0) & (b < 32)
        assert np.array_equal(hist.astype(np.int64), np.bincount(b[inr], minlength=32))
        assert cu == np.count_nonzero(b < 0) and co == np.count_nonzero(b >= 32)
    assert ctr[6] == N ** 3 and ctr[5] == 0
    assert qr.sum() + ctr[0] == N ** 3
    # moments are plain power sums
    assert mom[0] == pytest.approx((A[0, 0] ** 2).sum(), rel=1e-13)
    assert mom[4 * 5 + 3] == pytest.approx((A[1, 2] ** 6).sum(), rel=1e-13)
    assert mom[38] == pytest.approx(eps.sum(), rel=1e-13)
    assert mom[43] == pytest.approx((ens ** 2).sum(), rel=1e-13)


def test_gradient_component_histograms_against_brute_force():
    """Longitudinal (A_11, A_22, A_33) and transverse (A_ij, i != j)
    components pooled, in units of sqrt(q0), against independent binning;
    every point contributes 3 + 6 samples."""
    N = 8
    m = O.Member(N=N, nu=0.05, seed=9, init_energy=3.0)
    uh = O.initial_field(m)
    h = O.HistSpec(qr_bins=8, q_lim=4.0, r_lim=4.0, tail_bins=16, tail_lo=-3.0, tail_hi=2.0,
                   eps_norm=0.1, nu_norm=0.05, grad_bins=24, grad_lim=3.0)
    assert h.counts_len == 64 + 32 + 8 + 48 + 4
    counts, _ = O.gradient_stats(uh, m.nu, h)
    lon, tra, gc = O.split_grad_counts(counts, h)
    A = O.gradient(uh)
    g0 = np.sqrt(h.eps_norm / (2 * h.nu_norm))
    eg = np.array([np.float32(-3.0 + 6.0 * b / 24) for b in range(25)], dtype=np.float32)
    for comps, hist, cu, co in (([(0, 0), (1, 1), (2, 2)], lon, gc[0], gc[1]),
                                ([(0, 1), (0, 2), (1, 0), (1, 2), (2, 0), (2, 1)], tra, gc[2], gc[3])):
        b = np.concatenate([brute_bins((A[i, j] / g0).ravel(), eg) for i, j in comps])
        inr = (b >= 0) & (b < 24)
        assert np.array_equal(hist.astype(np.int64), np.bincount(b[inr], minlength=24))
        assert cu == np.count_nonzero(b < 0) and co == np.count_nonzero(b >= 24)
        assert hist.sum() + cu + co == len(comps) * N ** 3
    # the first part of the layout is unchanged by the gradient histograms
    h0 = O.HistSpec(qr_bins=8, q_lim=4.0, r_lim=4.0, tail_bins=16, tail_lo=-3.0, tail_hi=2.0,
                    eps_norm=0.1, nu_norm=0.05)
    c0, _ = O.gradient_stats(uh, m.nu, h0)
    assert np.array_equal(c0, counts[: h0.counts_len])


def test_log_histogram_underflow_for_zero():
    """A field at rest has eps = omega^2 = 0: every point is underflow."""
    N = 4
    uh = np.zeros((3, N, N, N // 2 + 1), dtype=complex)
    h = O.HistSpec(qr_bins=8, tail_bins=8, nu_norm=0.1)
    counts, _ = O.gradient_stats(uh, 0.1, h)
    qr, he, hw, ctr = O.split_counts(counts, h)
    assert ctr[1] == N ** 3 and ctr[3] == N ** 3 and he.sum() == 0 and hw.sum() == 0
    # Q = R = 0 lies in the interior bins of a symmetric axis
    assert qr[4, 4] == N ** 3


def test_bin_rule_on_edges_against_searchsorted():
    """The oracle's bin rule on probe values at and beside every FP32 edge,
    signed zeros, subnormals, the FP32 extremes and infinities, against
    numpy's searchsorted on the same edges (edge[b] <= x < edge[b+1]; -1
    below, n at or above the last edge; a non-positive value on the log
    axis is underflow)."""
    h = O.HistSpec(qr_bins=64, q_lim=10.0, r_lim=7.5, tail_bins=256, tail_lo=-8.0, tail_hi=8.0,
                   eps_norm=0.1, nu_norm=0.005, grad_bins=96, grad_lim=40.0)
    axes = {
        0: np.array([-10.0 + 20.0 * b / 64 for b in range(65)], dtype=np.float32),
        1: np.array([-7.5 + 15.0 * b / 64 for b in range(65)], dtype=np.float32),
        2: np.array([10.0 ** (-8.0 + 16.0 * b / 256) for b in range(257)], dtype=np.float32),
        3: np.array([-40.0 + 80.0 * b / 96 for b in range(97)], dtype=np.float32),
    }
    for axis, e in axes.items():
        x = I.bin_probe_values(e, seed=axis, log=axis == 2)
        got = O.bin_values(h, axis, x)
        ref = brute_bins(x, e)
        ref = np.where(ref >= len(e) - 1, len(e) - 1, ref)
        if axis == 2:
            ref = np.where(x > 0, ref, -1)
        assert np.array_equal(got, ref), axis
        # every edge opens its own bin, its lower neighbour closes the one before
        nb = len(e) - 1
        assert np.array_equal(got[: nb + 1], np.arange(nb + 1))
        assert np.array_equal(got[2 * (nb + 1): 3 * (nb + 1)], np.arange(-1, nb))
