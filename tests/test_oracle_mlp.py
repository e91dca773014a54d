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


# ---------------------------------------------------------------------------
# forward pass pinned to hand-evaluated values (independent of the oracle's
# own loss): the constants below were evaluated once at 30 digits from
# sigma(z) = 1 / (1 + e^-z), SiLU(z) = z sigma(z), and written in as numbers
# ---------------------------------------------------------------------------
Q_HARM_M05 = [-1.0, 0.0, 0.0, -1.0, 1.0, 0.0, 0.0, 1.0]   # sin/cos(pi k s), k = 1..4, at s = -0.5
HARM_0 = [0.0, 1.0] * 4                                   # at s = 0
HARM_P05 = [1.0, 0.0, 0.0, -1.0, -1.0, 0.0, 0.0, 1.0]     # at s = +0.5


def test_feature_rows_hand_written():
    """Rows of a 2 x 2 joint grid and 2-bin tails at lambda = 0.5: bin
    coordinates, lambda / 5, the one-hot kind, and the eight harmonics of each
    coordinate in the documented order; zeros from input 31 on."""
    F = M.features(0.5, 2, 2)
    assert F.shape == (4 + 4, 64)
    pad = [0.0] * (64 - 31)
    row_qr0 = [-0.5, -0.5, 0.1, 0.0, 1.0, 0.0, 0.0] + Q_HARM_M05 + Q_HARM_M05 + HARM_0 + pad
    row_eps0 = [0.0, 0.0, 0.1, -0.5, 0.0, 1.0, 0.0] + HARM_0 + HARM_0 + Q_HARM_M05 + pad
    row_ens1 = [0.0, 0.0, 0.1, 0.5, 0.0, 0.0, 1.0] + HARM_0 + HARM_0 + HARM_P05 + pad
    np.testing.assert_allclose(F[0], row_qr0, atol=1e-15)
    np.testing.assert_allclose(F[4], row_eps0, atol=1e-15)
    np.testing.assert_allclose(F[7], row_ens1, atol=1e-15)
    # joint bin 1 is (q, r) = (-0.5, +0.5): row-major over (Q, R)
    assert F[1, 0] == -0.5 and F[1, 1] == 0.5


def test_silu_known_values():
    z = np.array([1.0, -1.0, 2.0, -3.0, 0.5, 0.0])
    ref = [0.73105857863000487925, -0.26894142136999512075, 1.7615941559557648881, -0.14227761953270034264,
           0.31122966560092728232, 0.0]
    np.testing.assert_allclose(M.silu(z), ref, rtol=1e-15, atol=0)


def _net(entries):
    _, n = M.layout()
    g = M.unpack(np.zeros(n))
    for (name, idx), v in entries.items():
        g[name][idx] = v
    return M.pack(g)


def test_forward_chain_through_three_layers():
    """One hidden unit carries lambda (W1 picks input 2, lambda / 5, times 5)
    through the three SiLU layers with biases and scalings at every layer;
    every other unit stays at SiLU(0) = 0, so the logit is the same for every
    bin and equals the hand-evaluated chain."""
    p = _net({("W1", (0, 2)): 5.0, ("b2", 0): -0.25, ("W2", (0, 0)): 1.0, ("W3", (0, 0)): 2.0,
              ("w4", 0): 3.0, ("b4", 0): 0.125})
    for lam, h1, h2, h3, logit in ((1.0, 0.73105857863000487925, 0.29729314880669161996, 0.38316137665813842256,
                                    1.2744841299744152677),
                                   (-2.0, -0.23840584404423511188, -0.18572569074987754461,
                                    -0.15162287433913631669, -0.32986862301740895006)):
        out, (F, z1, a1, z2, a2, z3, a3) = M.forward(p, M.features(lam, 2, 2))
        np.testing.assert_allclose(a1[:, 0], h1, rtol=1e-14)
        np.testing.assert_allclose(a2[:, 0], h2, rtol=1e-14)
        np.testing.assert_allclose(a3[:, 0], h3, rtol=1e-14)
        np.testing.assert_allclose(out, logit, rtol=1e-14)
        assert np.all(a1[:, 1:] == 0) and np.all(a3[:, 1:] == 0)


def test_densities_softmax_per_kind_closed_form():
    """Unit 0 carries 2q and unit 1 carries -x through the three layers
    (identity weights), w4 = (1, 1): joint bins with q = -0.5 and +0.5 get
    logits sss(-1) and sss(1), the tail bins sss(0.5) and sss(-0.5) (sss =
    SiLU applied three times); each kind is normalised on its own."""
    p = _net({("W1", (0, 0)): 2.0, ("W1", (1, 3)): -1.0, ("W2", (0, 0)): 1.0, ("W2", (1, 1)): 1.0,
              ("W3", (0, 0)): 1.0, ("W3", (1, 1)): 1.0, ("w4", 0): 1.0, ("w4", 1): 1.0})
    q = M.densities(p, [0.3], 2, 2)[0]
    a, b = 0.20532456273179496587, 0.29467543726820503413     # q = -0.5 (bins 0, 1), q = +0.5 (bins 2, 3)
    c, d = 0.53464172855360363263, 0.46535827144639636737     # tail x = -0.5 (bin 0), x = +0.5 (bin 1)
    np.testing.assert_allclose(q, [a, a, b, b, c, d, c, d], rtol=1e-13)
    logit, _ = M.forward(p, M.features(0.3, 2, 2))
    np.testing.assert_allclose(logit[[0, 2, 4, 5]], [-0.054859244007100535191, 0.30642333401972688772,
                                                     0.097864364047002523355, -0.040924907115727866827], rtol=1e-13)
