"""Pin of the oracle MLP gradient: central finite differences of its own
loss (no GPU)."""
import numpy as np

import oracle.mlp as M


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    _, n = M.layout()
    p = rng.standard_normal(n) * 0.05
    nq, nt = 3, 4
    L = nq * nq + 2 * nt + 8
    counts = rng.integers(0, 20, size=(2, L))
    lams = [-0.7, 1.3]
    f0, g = M.loss_grad(p, lams, counts, nq, nt)
    assert np.isfinite(f0) and f0 > 0
    lay, _ = M.layout()
    picks = []
    for k, (o, m) in lay.items():
        picks += list(o + rng.choice(m, size=min(m, 6), replace=False))
    h = 1e-6
    for i in picks:
        e = np.zeros(n)
        e[i] = h
        fd = (M.loss_grad(p + e, lams, counts, nq, nt)[0] - M.loss_grad(p - e, lams, counts, nq, nt)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_features_and_densities():
    F = M.features(0.5, 4, 6)
    assert F.shape == (16 + 12, 64)
    # kind one-hot and lambda/5
    assert np.all(F[:16, 4] == 1) and np.all(F[16:22, 5] == 1) and np.all(F[22:, 6] == 1)
    assert np.allclose(F[:, 2], 0.1)
    assert np.all(F[:, 31:] == 0)
    _, n = M.layout()
    q = M.densities(np.random.default_rng(1).standard_normal(n) * 0.1, [0.0, 1.0], 4, 6)
    assert np.allclose(q[:, :16].sum(axis=1), 1) and np.allclose(q[:, 16:22].sum(axis=1), 1)
