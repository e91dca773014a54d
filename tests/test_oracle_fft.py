"""Pins of the oracle FFT against brute-force DFTs (no GPU).

The oracle's own recursive mixed-radix FFT must agree with the O(N^2) /
O(N^6) definition of the discrete Fourier transform; angles in the brute
force are reduced modulo n before the exponential so that the reference
itself is accurate to rounding.
"""
import numpy as np
import pytest

import oracle as O


def dft_matrix(n, sign=-1):
    j = np.arange(n)
    return np.exp(sign * 2j * np.pi * (np.outer(j, j) % n) / n)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 8, 9, 12, 16, 18, 24, 27, 32, 48, 64, 96, 5, 7, 10])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft1_matches_brute_force(n, sign):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = dft_matrix(n, sign) @ x
    got = O.fft1(x, sign)
    assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("N", [6, 8])
def test_rfft3_matches_brute_force_dft(N):
    """Forward transform = N^-3 sum_x u(x) exp(-i k.x), brute force O(N^6)."""
    rng = np.random.default_rng(N)
    u = rng.standard_normal((N, N, N))
    W = dft_matrix(N)
    full = np.einsum("ax,by,cz,xyz->abc", W, W, W, u) / N ** 3
    got = O.rfft3(u)
    assert got.shape == (N, N, N // 2 + 1)
    assert np.abs(got - full[:, :, : N // 2 + 1]).max() < 1e-13


@pytest.mark.parametrize("N", [6, 8, 12])
def test_irfft3_is_synthesis_and_inverse(N):
    """Inverse = sum_k uh_k exp(i k.x) over the Hermitian-completed spectrum."""
    rng = np.random.default_rng(100 + N)
    u = rng.standard_normal((N, N, N))
    uh = O.rfft3(u)
    back = O.irfft3(uh)
    assert np.abs(back - u).max() < 1e-13
    # synthesis of a single mode: uh at (1, 2, 1) and its Hermitian image
    uh = np.zeros((N, N, N // 2 + 1), dtype=complex)
    uh[1, 2, 1] = 0.3 - 0.2j
    x = 2 * np.pi * np.arange(N) / N
    X, Y, Zz = np.meshgrid(x, x, x, indexing="ij")
    ref = 2 * np.real((0.3 - 0.2j) * np.exp(1j * (X + 2 * Y + Zz)))
    assert np.abs(O.irfft3(uh) - ref).max() < 1e-13


def test_irfft3_drops_imaginary_part_of_kz0_mean():
    """kz = 0 plane enters through Hermitian completion: an imaginary mean
    mode contributes nothing to the real field."""
    N = 8
    uh = np.zeros((N, N, N // 2 + 1), dtype=complex)
    uh[0, 0, 0] = 1.0 + 5.0j
    assert np.abs(O.irfft3(uh) - 1.0).max() < 1e-15
