"""FP64 CPU oracle of the ensemble DNS hot path.

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow restatement of the
method of Bentkamp & Wilczek (ensemble hypothesis, Sec. II; Gaussian lambda
weights, Sec. IV; member DNS, Sec. IV; gradient statistics, Secs. V-VII),
written to check the CUDA library against.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  It shares no code with the CUDA path and never imports the product
package.

The C part (``fft.c``, ``ns.c``, ``stats.c``) is compiled by :func:`build`
with gcc into ``liboracle.so`` beside the sources; this module wraps it with
numpy arrays.  The weight and mixture arithmetic lives in ``mixture.py`` and
the FP64 reference MLP in ``mlp.py``.

Parity pins: every function here is checked by ``tests/test_oracle_*.py``
against closed forms, brute force or values the paper prints.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SOURCES = ("fft.c", "ns.c", "stats.c")
_lib = None

NMOM = 48


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, FP64, OpenMP, no fast-math)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_SO):
        so_time = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= so_time for s in srcs):
            return _SO
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-Wall",
           "-o", _SO + ".tmp"] + [os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


class _Member(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("rk_order", ctypes.c_int), ("nu", ctypes.c_double),
                ("lam", ctypes.c_double), ("eps_bar", ctypes.c_double), ("k_lo", ctypes.c_double),
                ("k_hi", ctypes.c_double), ("dt", ctypes.c_double), ("cfl", ctypes.c_double),
                ("dt_max", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("init_energy", ctypes.c_double)]


class _Diag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("t", "dt", "E", "diss", "EB", "P", "umax")]


class _HistSpec(ctypes.Structure):
    _fields_ = [("qr_bins", ctypes.c_int), ("q_lim", ctypes.c_double), ("r_lim", ctypes.c_double),
                ("tail_bins", ctypes.c_int), ("tail_lo", ctypes.c_double),
                ("tail_hi", ctypes.c_double), ("eps_norm", ctypes.c_double),
                ("nu_norm", ctypes.c_double), ("grad_bins", ctypes.c_int), ("grad_lim", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.POINTER
        d, i = ctypes.c_double, ctypes.c_int
        vp = ctypes.c_void_p
        L.or_fft1.argtypes = [vp, i, i]
        L.or_rfft3.argtypes = [vp, vp, i]
        L.or_irfft3.argtypes = [vp, vp, i]
        L.or_kc.argtypes = [i]
        L.or_kc.restype = i
        L.or_band_modes.argtypes = [i, d, d]
        L.or_band_modes.restype = i
        L.or_initial_field.argtypes = [P(_Member), vp]
        L.or_white_noise.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.or_white_noise.restype = d
        L.or_rhs.argtypes = [P(_Member), vp, vp, vp, P(d), P(d)]
        L.or_sums.argtypes = [P(_Member), vp, P(d), P(d), P(d)]
        L.or_step.argtypes = [P(_Member), vp, i, P(d), P(_Diag)]
        L.or_step.restype = i
        L.or_counts_len.argtypes = [P(_HistSpec)]
        L.or_counts_len.restype = i
        L.or_gradient.argtypes = [vp, i, vp]
        L.or_invariants.argtypes = [vp, i, d, vp, vp, vp, vp]
        L.or_gradient_stats.argtypes = [vp, i, d, P(_HistSpec), vp, vp]
        L.or_bin_values.argtypes = [P(_HistSpec), i, vp, ctypes.c_long, vp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# member description and histogram specification
# ---------------------------------------------------------------------------
@dataclass
class Member:
    N: int
    nu: float
    lam: float = 0.0
    eps_bar: float = 0.1
    k_lo: float = 1.0
    k_hi: float = 2.0
    dt: float = 0.01
    cfl: float = 0.2
    dt_max: float = 0.0
    rk_order: int = 2
    seed: int = 0
    init_energy: float = 0.5

    def _c(self) -> _Member:
        return _Member(self.N, self.rk_order, self.nu, self.lam, self.eps_bar, self.k_lo, self.k_hi,
                       self.dt, self.cfl, self.dt_max, self.seed, self.init_energy)


@dataclass
class HistSpec:
    qr_bins: int = 64
    q_lim: float = 10.0
    r_lim: float = 10.0
    tail_bins: int = 256
    tail_lo: float = -8.0
    tail_hi: float = 8.0
    eps_norm: float = 0.1
    nu_norm: float = 0.02
    grad_bins: int = 0
    grad_lim: float = 40.0

    def _c(self) -> _HistSpec:
        return _HistSpec(self.qr_bins, self.q_lim, self.r_lim, self.tail_bins, self.tail_lo,
                         self.tail_hi, self.eps_norm, self.nu_norm, self.grad_bins, self.grad_lim)

    @property
    def counts_len(self) -> int:
        g = 2 * self.grad_bins + 4 if self.grad_bins > 0 else 0
        return self.qr_bins ** 2 + 2 * self.tail_bins + 8 + g


# ---------------------------------------------------------------------------
# FFT
# ---------------------------------------------------------------------------
def fft1(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised complex DFT of a 1D array (own FFT)."""
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    lib().or_fft1(_ptr(a), a.size, sign)
    return a


def rfft3(u: np.ndarray) -> np.ndarray:
    """Forward 3D transform of a real [N,N,N] field, normalised by N^-3."""
    N = u.shape[0]
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty((N, N, N // 2 + 1), dtype=np.complex128)
    lib().or_rfft3(_ptr(u), _ptr(out), N)
    return out


def irfft3(uh: np.ndarray) -> np.ndarray:
    """Inverse 3D transform (synthesis) of an [N,N,N/2+1] half spectrum."""
    N = uh.shape[0]
    uh = np.ascontiguousarray(uh, dtype=np.complex128)
    out = np.empty((N, N, N), dtype=np.float64)
    lib().or_irfft3(_ptr(uh), _ptr(out), N)
    return out


# ---------------------------------------------------------------------------
# solver
# ---------------------------------------------------------------------------
def kc(N: int) -> int:
    return lib().or_kc(N)


def band_modes(N: int, k_lo: float, k_hi: float) -> int:
    return lib().or_band_modes(N, k_lo, k_hi)


def white_noise(seed: int, counter: int) -> float:
    return lib().or_white_noise(seed, counter)


def initial_field(m: Member) -> np.ndarray:
    """Seeded initial spectral field, shape [3, N, N, N/2+1]."""
    N = m.N
    out = np.zeros((3, N, N, N // 2 + 1), dtype=np.complex128)
    mc = m._c()
    lib().or_initial_field(ctypes.byref(mc), _ptr(out))
    return out


def rhs(m: Member, uh: np.ndarray):
    """F(uh) = P N(uh) + f(uh); returns (F, projected nonlinear term, umax, alpha)."""
    uh = np.ascontiguousarray(uh, dtype=np.complex128)
    F = np.zeros_like(uh)
    nl = np.zeros_like(uh)
    umax, alpha = ctypes.c_double(), ctypes.c_double()
    mc = m._c()
    lib().or_rhs(ctypes.byref(mc), _ptr(uh), _ptr(F), _ptr(nl), ctypes.byref(umax),
                 ctypes.byref(alpha))
    return F, nl, umax.value, alpha.value


def sums(m: Member, uh: np.ndarray):
    """(E, dissipation, band energy) of a spectral state."""
    uh = np.ascontiguousarray(uh, dtype=np.complex128)
    E, D, B = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    mc = m._c()
    lib().or_sums(ctypes.byref(mc), _ptr(uh), ctypes.byref(E), ctypes.byref(D), ctypes.byref(B))
    return E.value, D.value, B.value


def step(m: Member, uh: np.ndarray, nsteps: int, t: float = 0.0):
    """Advance nsteps in place; returns (status, diag dict)."""
    assert uh.dtype == np.complex128 and uh.flags["C_CONTIGUOUS"]
    tt = ctypes.c_double(t)
    d = _Diag()
    mc = m._c()
    st = lib().or_step(ctypes.byref(mc), _ptr(uh), nsteps, ctypes.byref(tt), ctypes.byref(d))
    return st, {k: getattr(d, k) for k, _ in _Diag._fields_}


# ---------------------------------------------------------------------------
# gradient statistics
# ---------------------------------------------------------------------------
def gradient(uh: np.ndarray) -> np.ndarray:
    """A_ij = d_j u_i as [3, 3, N, N, N]."""
    N = uh.shape[1]
    uh = np.ascontiguousarray(uh, dtype=np.complex128)
    A = np.empty((3, 3, N, N, N), dtype=np.float64)
    lib().or_gradient(_ptr(uh), N, _ptr(A))
    return A


def invariants(A: np.ndarray, nu: float):
    """(Q, R, eps, omega^2) fields from the gradient tensor fields."""
    N = A.shape[2]
    A = np.ascontiguousarray(A, dtype=np.float64)
    outs = [np.empty((N, N, N), dtype=np.float64) for _ in range(4)]
    lib().or_invariants(_ptr(A), N, nu, *[_ptr(o) for o in outs])
    return tuple(outs)


def gradient_stats(uh: np.ndarray, nu: float, h: HistSpec, counts=None, moments=None):
    """Accumulate one snapshot's histograms and moments (in place if given)."""
    N = uh.shape[1]
    uh = np.ascontiguousarray(uh, dtype=np.complex128)
    if counts is None:
        counts = np.zeros(h.counts_len, dtype=np.uint64)
    if moments is None:
        moments = np.zeros(NMOM, dtype=np.float64)
    hc = h._c()
    lib().or_gradient_stats(_ptr(uh), N, nu, ctypes.byref(hc), _ptr(counts), _ptr(moments))
    return counts, moments


def bin_values(h: HistSpec, axis: int, x) -> np.ndarray:
    """The histogram bin rule on FP32 values already in an axis's units
    (0 Q/q0, 1 R/q0^1.5, 2 the log10 tail axis, 3 A_ij/sqrt(q0)): -1 for
    underflow, the axis's bin count for overflow."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.size, dtype=np.int32)
    hc = h._c()
    lib().or_bin_values(ctypes.byref(hc), axis, _ptr(x), x.size, _ptr(out))
    return out


def split_counts(counts: np.ndarray, h: HistSpec):
    """View a counts vector as (qr [nq, nq], eps [nt], ens [nt], counters [8])."""
    nq, nt = h.qr_bins, h.tail_bins
    qr = counts[: nq * nq].reshape(nq, nq)
    e = counts[nq * nq: nq * nq + nt]
    w = counts[nq * nq + nt: nq * nq + 2 * nt]
    c = counts[nq * nq + 2 * nt: nq * nq + 2 * nt + 8]
    return qr, e, w, c


def split_grad_counts(counts: np.ndarray, h: HistSpec):
    """View the gradient-component part of a counts vector as (longitudinal
    [ng], transverse [ng], counters [4]: long_under, long_over, trans_under,
    trans_over)."""
    off = h.qr_bins ** 2 + 2 * h.tail_bins + 8
    ng = h.grad_bins
    return counts[off: off + ng], counts[off + ng: off + 2 * ng], counts[off + 2 * ng: off + 2 * ng + 4]
