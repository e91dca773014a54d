"""Oracle of the learned lambda interpolant: FP64 MLP forward, loss and
gradient in numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The paper mixes
member statistics directly (Sec. II, Eq. ensemble_hypothesis; Sec. IV); the
interpolant is this implementation's addition, specified in include/ens.h:

  rows      one per (member lambda, bin) for the joint Q-R bins, then the
            dissipation bins, then the enstrophy bins
  features  bin coordinates scaled to [-1, 1] (Q, R for the joint PDF; the
            log axis for the tails), lambda / 5, one-hot PDF kind, and
            sin/cos(pi k s) of the three coordinates for k = 1..4 (31 used of
            64 inputs)
  network   z1 = W1 f + b1, h1 = SiLU(z1), z2 = W2 h1 + b2, h2 = SiLU(z2),
            z3 = W3 h2 + b3, h3 = SiLU(z3), logit = w4 . h3 + b4
  loss      mean over (member, kind) of -sum_b p_b log softmax(logit)_b,
            p = the member's in-range histogram of that kind, unit sum
  params    W1 [256][64], b1, W2 [256][256], b2, W3 [256][256], b3, w4, b4

Pinned by ``tests/test_oracle_mlp.py`` against central finite differences.
"""
from __future__ import annotations

import math

import numpy as np

HID, NIN = 256, 64


def layout():
    sizes = [("W1", HID * NIN), ("b1", HID), ("W2", HID * HID), ("b2", HID), ("W3", HID * HID), ("b3", HID),
             ("w4", HID), ("b4", 1)]
    out, o = {}, 0
    for k, n in sizes:
        out[k] = (o, n)
        o += n
    return out, o


def unpack(p):
    L, _ = layout()
    g = {k: np.asarray(p[o:o + n], dtype=np.float64) for k, (o, n) in L.items()}
    g["W1"] = g["W1"].reshape(HID, NIN)
    g["W2"] = g["W2"].reshape(HID, HID)
    g["W3"] = g["W3"].reshape(HID, HID)
    return g


def pack(g):
    L, total = layout()
    p = np.zeros(total, dtype=np.float64)
    for k, (o, n) in L.items():
        p[o:o + n] = np.asarray(g[k], dtype=np.float64).ravel()
    return p


def features(lam, nq, nt):
    """Feature rows [nq*nq + 2 nt, 64] of one lambda value."""
    rows = []
    for b in range(nq * nq + 2 * nt):
        q = r = x = 0.0
        if b < nq * nq:
            kind = 0
            q = ((b // nq) + 0.5) / nq * 2.0 - 1.0
            r = ((b % nq) + 0.5) / nq * 2.0 - 1.0
        else:
            bb = b - nq * nq
            kind = 1 if bb < nt else 2
            x = ((bb % nt) + 0.5) / nt * 2.0 - 1.0
        f = [q, r, lam / 5.0, x, 0.0, 0.0, 0.0]
        f[4 + kind] = 1.0
        for s in (q, r, x):
            for k in range(1, 5):
                f += [math.sin(math.pi * k * s), math.cos(math.pi * k * s)]
        f += [0.0] * (NIN - len(f))
        rows.append(f)
    return np.array(rows, dtype=np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def targets(counts, nq, nt):
    """Per member, the three normalised in-range histograms, concatenated."""
    counts = np.asarray(counts, dtype=np.float64)
    out = []
    for c in counts:
        parts = [c[:nq * nq], c[nq * nq:nq * nq + nt], c[nq * nq + nt:nq * nq + 2 * nt]]
        out.append(np.concatenate([p / p.sum() if p.sum() > 0 else p for p in parts]))
    return np.array(out)


def forward(p, F):
    g = unpack(p)
    z1 = F @ g["W1"].T + g["b1"]
    h1 = silu(z1)
    z2 = h1 @ g["W2"].T + g["b2"]
    h2 = silu(z2)
    z3 = h2 @ g["W3"].T + g["b3"]
    h3 = silu(z3)
    logit = h3 @ g["w4"] + g["b4"][0]
    return logit, (F, z1, h1, z2, h2, z3, h3)


def _groups(nq, nt):
    return [(0, nq * nq), (nq * nq, nq * nq + nt), (nq * nq + nt, nq * nq + 2 * nt)]


def densities(p, lams, nq, nt):
    """Softmax densities per lambda and kind: [len(lams), nq*nq + 2 nt]."""
    out = []
    for lam in lams:
        logit, _ = forward(p, features(lam, nq, nt))
        q = np.empty_like(logit)
        for a, b in _groups(nq, nt):
            z = logit[a:b] - logit[a:b].max()
            q[a:b] = np.exp(z) / np.exp(z).sum()
        out.append(q)
    return np.array(out)


def loss_grad(p, lams, counts, nq, nt):
    """Loss (mean cross-entropy over member-kind groups) and its gradient."""
    P = targets(counts, nq, nt)
    n = len(lams)
    w = 1.0 / (3.0 * n)
    grad = {k: 0.0 for k in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4")}
    g = unpack(p)
    total = 0.0
    for i, lam in enumerate(lams):
        logit, (F, z1, h1, z2, h2, z3, h3) = forward(p, features(lam, nq, nt))
        dlogit = np.zeros_like(logit)
        for a, b in _groups(nq, nt):
            z = logit[a:b] - logit[a:b].max()
            lq = z - math.log(np.exp(z).sum())
            pt = P[i, a:b]
            total += -w * float(np.sum(pt[pt > 0] * lq[pt > 0]))
            dlogit[a:b] = w * (np.exp(lq) - pt)
        grad["w4"] = grad["w4"] + h3.T @ dlogit
        grad["b4"] = grad["b4"] + dlogit.sum()
        dz3 = np.outer(dlogit, g["w4"]) * dsilu(z3)
        grad["W3"] = grad["W3"] + dz3.T @ h2
        grad["b3"] = grad["b3"] + dz3.sum(axis=0)
        dz2 = (dz3 @ g["W3"]) * dsilu(z2)
        grad["W2"] = grad["W2"] + dz2.T @ h1
        grad["b2"] = grad["b2"] + dz2.sum(axis=0)
        dz1 = (dz2 @ g["W2"]) * dsilu(z1)
        grad["W1"] = grad["W1"] + dz1.T @ F
        grad["b1"] = grad["b1"] + dz1.sum(axis=0)
    grad["b4"] = np.array([grad["b4"]])
    return total, pack(grad)
