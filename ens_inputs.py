"""Seeded synthetic inputs and workload descriptions shared by the tests and
the benchmark.

This module holds no arithmetic of the method: it only draws seeded random
numbers and lists member parameters.  Both the oracle and the CUDA path take
their inputs from here; neither imports the other.

Workloads (shapes of the paper's ensembles, Sec. IV, Table I: ens256 has 48
members on 256^3 grids with lambda in [-5.1, 5.8]):
  single_member_32 : 1 member, 32^3, nu = 0.02, band [1, 2], eps_bar = 0.1,
                     IF-RK2, dt = 0.01, seed 0, E0 = 0.5
  ensemble_64      : 16 members, 64^3, nu = 0.01, band [3, 5], lambda on a
                     uniform grid over [-3, 3], IF-RK3, CFL 0.2 (dt <= 0.01)
  ensemble_256     : 64 members, 256^3, nu = 0.005, band [6, 8], lambda from
                     N(0, 2^2) (Philox counter generator, key 2026) clipped
                     to [-5.1, 5.8], IF-RK3, CFL 0.2
  uneven_batch     : 24 x 128^3, 12 x 256^3, 4 x 384^3, lambda on [-2, 2],
                     viscosity per member so that k_max eta >= 1.5
"""
from __future__ import annotations

import math

import numpy as np


def kept_mask(N: int) -> np.ndarray:
    """Support of a dealiased half spectrum [N, N, N/2+1]: max_i |k_i| <= ceil(N/3) - 1."""
    kc = (N + 2) // 3 - 1
    k = np.fft.fftfreq(N, 1.0 / N)
    kz = np.arange(N // 2 + 1)
    KX, KY, KZ = np.meshgrid(k, k, kz, indexing="ij")
    return (np.abs(KX) <= kc) & (np.abs(KY) <= kc) & (KZ <= kc)


def random_spectral(N: int, seed: int, scale: float = 1e-3) -> np.ndarray:
    """Complex normal values on the dealiased support, [3, N, N, N/2+1]."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    shape = (3, N, N, N // 2 + 1)
    out = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * scale
    out[:, ~kept_mask(N)] = 0.0
    return out


def random_physical(N: int, seed: int) -> np.ndarray:
    """Real standard normal values, [3, N, N, N]."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    return rng.standard_normal((3, N, N, N))


def cosine_modes(N: int, modes) -> np.ndarray:
    """Physical field sum of a cos(k.x) for (component, k, a) in modes."""
    x = 2 * np.pi * np.arange(N) / N
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    u = np.zeros((3, N, N, N))
    for comp, (kx, ky, kz), a in modes:
        u[comp] += a * np.cos(kx * X + ky * Y + kz * Z)
    return u


def abc_flow(N: int, A: float = 1.0, B: float = 0.7, C: float = 0.4) -> np.ndarray:
    x = 2 * np.pi * np.arange(N) / N
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    return np.stack([A * np.sin(Z) + C * np.cos(Y), B * np.sin(X) + A * np.cos(Z), C * np.sin(Y) + B * np.cos(X)])


def synthetic_member_counts(lams, nq, nt, npoints, seed):
    """Member histograms drawn from smooth, lambda-dependent model densities
    (multinomial samples of npoints per PDF kind), in the library's counts
    layout [qr nq*nq | eps nt | enstrophy nt | 8 counters]; npoints is stored
    at counter 6.  Used to exercise the lambda interpolant on inputs with a
    known smooth lambda dependence."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    c = (np.arange(nq) + 0.5) / nq * 2 - 1
    Qg, Rg = np.meshgrid(c, c, indexing="ij")
    x = (np.arange(nt) + 0.5) / nt * 2 - 1
    out = np.zeros((len(lams), nq * nq + 2 * nt + 8), dtype=np.uint64)
    for i, lam in enumerate(lams):
        s = 0.25 * math.exp(lam / 8.0)
        pqr = np.exp(-(Qg ** 2 + (Rg - 0.2 * Qg) ** 2) / (2 * s * s)) * (1 + 0.3 * np.tanh(3 * (Rg + Qg)))
        pe = np.exp(-(x - (-0.2 + 0.08 * lam)) ** 2 / (2 * (0.15 * math.exp(lam / 10.0)) ** 2))
        pw = np.exp(-(x - (-0.1 + 0.1 * lam)) ** 2 / (2 * (0.18 * math.exp(lam / 10.0)) ** 2))
        parts = []
        for p in (pqr.ravel(), pe, pw):
            p = p / p.sum()
            parts.append(rng.multinomial(npoints, p))
        out[i, :nq * nq] = parts[0]
        out[i, nq * nq:nq * nq + nt] = parts[1]
        out[i, nq * nq + nt:nq * nq + 2 * nt] = parts[2]
        out[i, nq * nq + 2 * nt + 6] = npoints
    return out


# ---------------------------------------------------------------------------
# workloads: lists of member parameter dicts (keys of ens_member_desc)
# ---------------------------------------------------------------------------
def single_member_32():
    return [dict(N=32, nu=0.02, lam=0.0, eps_bar=0.1, k_lo=1.0, k_hi=2.0, dt=0.01, cfl=0.2, dt_max=0.0,
                 rk_order=2, seed=0, init_energy=0.5)]


def ensemble_64(n=16):
    lams = np.linspace(-3.0, 3.0, n)
    return [dict(N=64, nu=0.01, lam=float(l), eps_bar=0.1, k_lo=3.0, k_hi=5.0, dt=-1.0, cfl=0.2, dt_max=0.01,
                 rk_order=3, seed=i, init_energy=0.5) for i, l in enumerate(lams)]


def ensemble_256_lambdas(n=64, key=2026):
    rng = np.random.Generator(np.random.Philox(key=key))
    return np.clip(2.0 * rng.standard_normal(n), -5.1, 5.8)


def ensemble_256(n=64, N=256):
    lams = ensemble_256_lambdas(n)
    return [dict(N=N, nu=0.005, lam=float(l), eps_bar=0.1, k_lo=6.0, k_hi=8.0, dt=-1.0, cfl=0.2, dt_max=0.0,
                 rk_order=3, seed=1000 + i, init_energy=0.5) for i, l in enumerate(lams)]


def mixed_resolution(n=64, lam_min=3.2, N_hi=512):
    """ensemble_256 with every member at lambda >= lam_min replaced by the
    same member on an N_hi grid (twice the small-scale resolution), as the
    paper does for its extreme-gradient predictions (Sec. VI)."""
    out = ensemble_256(n)
    for d in out:
        if d["lam"] >= lam_min:
            d["N"] = N_hi
    return out


def reference_512():
    """One 512^3 member at nu = 0.0015 forced at 1 <= |k| <= 2 with injection
    rate 0.1 (lambda = 0): the single-reference-run shape."""
    return [dict(N=512, nu=0.0015, lam=0.0, eps_bar=0.1, k_lo=1.0, k_hi=2.0, dt=-1.0, cfl=0.2, dt_max=0.0,
                 rk_order=3, seed=77, init_energy=0.5)]


def uneven_batch(counts=((128, 24), (256, 12), (384, 4))):
    out = []
    seed = 0
    for N, n in counts:
        lams = np.linspace(-2.0, 2.0, n)
        kmax = N / 3.0
        for l in lams:
            eps = 0.1 * math.exp(float(l))
            # k_max eta >= 1.5 with eta = (nu^3/eps)^(1/4): nu >= (1.5/k_max)^(4/3) eps^(1/3)
            nu = (1.5 / kmax) ** (4.0 / 3.0) * eps ** (1.0 / 3.0)
            out.append(dict(N=N, nu=nu, lam=float(l), eps_bar=0.1, k_lo=6.0, k_hi=8.0, dt=-1.0, cfl=0.2,
                            dt_max=0.0, rk_order=3, seed=seed, init_energy=0.5))
            seed += 1
    return out


def bin_probe_values(edges, n_random: int = 4096, seed: int = 0, log: bool = False) -> np.ndarray:
    """FP32 probe values for a histogram bin rule on the given FP32 edges:
    every edge and its FP32 neighbours on both sides, signed zeros, the
    smallest subnormals, the extremes of the FP32 range, infinities, and
    seeded values spread over the axis widened by one bin on each side
    (uniform, or log-uniform for a log axis)."""
    e = np.asarray(edges, dtype=np.float32)
    up = np.nextafter(e, np.float32(np.inf))
    dn = np.nextafter(e, np.float32(-np.inf))
    fmax = np.finfo(np.float32).max
    tiny = np.finfo(np.float32).tiny
    sub = np.float32(1.4e-45)
    specials = np.array([0.0, -0.0, sub, -sub, tiny, -tiny, fmax, -fmax, np.inf, -np.inf], dtype=np.float32)
    rng = np.random.default_rng(seed)
    nb = len(e) - 1
    if log:
        lo, hi = math.log10(float(e[0])), math.log10(float(e[-1]))
        pad = (hi - lo) / nb
        r = (10.0 ** rng.uniform(lo - pad, hi + pad, n_random)).astype(np.float32)
    else:
        lo, hi = float(e[0]), float(e[-1])
        pad = (hi - lo) / nb
        r = rng.uniform(lo - pad, hi + pad, n_random).astype(np.float32)
    return np.concatenate([e, up, dn, specials, r])
