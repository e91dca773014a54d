"""The learned lambda interpolant on the GPU (tcgen05 BF16 training and
inference kernels) against the FP64 oracle MLP, the member-quadrature
mixture, and the method without it.

Gradients: BF16 weights and activations with FP32 accumulation against FP64
on the same (BF16-rounded) weights: relative L2 <= 3e-2, cosine >= 0.999.
Mixture: Hellinger distance <= 0.02 to the member quadrature, per PDF.
"""
import numpy as np
import pytest

import ens_inputs as I
import oracle.mixture as OM
import oracle.mlp as OMLP

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


def bf16_round(x):
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint32) << 16
    return r.view(np.float32)


def bf16_params(p):
    """The parameters as the tensor-core path sees them: weight matrices and
    head rounded to BF16, biases in FP32."""
    lay, _ = OMLP.layout()
    q = p.astype(np.float64).copy()
    for k in ("W1", "W2", "W3"):
        o, n = lay[k]
        q[o:o + n] = bf16_round(p[o:o + n])
    return q


def hellinger_kinds(a, b, nq, nt):
    sl = [slice(0, nq * nq), slice(nq * nq, nq * nq + nt), slice(nq * nq + nt, nq * nq + 2 * nt)]
    return [OM.hellinger(a[s], b[s]) for s in sl]


def test_gradient_matches_oracle(E, parity_log):
    nq, nt = 8, 16
    h = E.hist_spec(qr_bins=nq, tail_bins=nt)
    lams = np.array([-1.2, 0.3, 2.0])
    counts = I.synthetic_member_counts(lams, nq, nt, 100000, seed=1)
    S = E.Surrogate(seed=7)
    p = S.params()
    loss, g = S.loss_grad(lams, counts, h)
    rl, rg = OMLP.loss_grad(bf16_params(p), lams, counts, nq, nt)
    assert loss == pytest.approx(rl, rel=2e-3)
    rel = np.linalg.norm(g - rg) / np.linalg.norm(rg)
    cos = float(g @ rg / (np.linalg.norm(g) * np.linalg.norm(rg)))
    parity_log("surrogate gradient (tcgen05 BF16) vs FP64 oracle MLP, rel L2", rel, 3e-2)
    parity_log("surrogate gradient, 1 - cosine", 1 - cos, 1e-3)
    assert rel < 3e-2 and cos > 0.999, (rel, cos)
    # per parameter block too
    lay, _ = OMLP.layout()
    for k, (o, n) in lay.items():
        if k == "b4":
            continue
        blk = np.linalg.norm(g[o:o + n] - rg[o:o + n]) / max(np.linalg.norm(rg[o:o + n]), 1e-30)
        assert blk < 5e-2, (k, blk)
    S.close()


def test_fused_inference_matches_layerwise_and_oracle(E, parity_log):
    """The fused inference kernel against the layer-by-layer forward pass
    (same BF16 roundings: logits to 1e-5 of their scale) and the FP64
    oracle MLP on the BF16-rounded weights (the kernel also rounds features
    and activations to BF16, ~0.4% each, so densities agree within 5% and
    Hellinger < 5e-3 per kind), over several 128-row tiles and a ragged
    last tile."""
    nq, nt = 16, 40            # 336 rows per lambda: tiles straddle lambda values
    h = E.hist_spec(qr_bins=nq, tail_bins=nt)
    lams = np.array([-2.7, -0.4, 0.9, 3.3, 5.1])
    counts = I.synthetic_member_counts(lams, nq, nt, 200000, seed=9)
    S = E.Surrogate(seed=11)
    S.train(lams, counts, h, 30, lr=2e-3)       # away from the initialisation
    lf = S.logits(lams, h, fused=True)
    ll = S.logits(lams, h, fused=False)
    assert np.abs(lf - ll).max() <= 1e-5 * max(1.0, np.abs(ll).max())
    q = S.density(lams, h)
    ref = OMLP.densities(bf16_params(S.params()), lams, nq, nt)
    assert np.all(np.abs(q - ref) <= 0.05 * ref + 1e-6)
    parity_log("surrogate densities (fused inference) vs FP64 oracle MLP, max Hellinger",
               max(max(hellinger_kinds(q[i], ref[i], nq, nt)) for i in range(len(lams))), 5e-3)
    for i in range(len(lams)):
        assert max(hellinger_kinds(q[i], ref[i], nq, nt)) < 5e-3
    S.close()


def trained(E, lams, counts, h, steps=1500, seed=3):
    S = E.Surrogate(seed=seed)
    l0, _ = S.loss_grad(lams, counts, h)
    l1 = S.train(lams, counts, h, steps, lr=2e-3)
    return S, l0, l1


def test_training_fits_members_and_mixture(E, parity_log):
    nq, nt = 16, 32
    h = E.hist_spec(qr_bins=nq, tail_bins=nt)
    lams = np.linspace(-3.0, 3.0, 16)
    counts = I.synthetic_member_counts(lams, nq, nt, 2_000_000, seed=2)
    S, l0, l1 = trained(E, lams, counts, h)
    assert l1 < l0
    q = S.density(lams, h)
    P = OMLP.targets(counts, nq, nt)
    worst = max(max(hellinger_kinds(q[i], P[i], nq, nt)) for i in range(len(lams)))
    assert worst < 0.03, worst
    # surrogate mixture on a 512-point lambda quadrature vs the member quadrature
    Z = 2.0
    moments = np.zeros((len(lams), 48))
    ref = E.ens_mixture_host(lams, counts, moments, h, kind=E.W_GAUSS_PAPER, c=0.023, Z=Z)
    d = lams[1] - lams[0]
    sur = S.mixture(h, lams[0] - d / 2, lams[-1] + d / 2, 512, kind=E.W_GAUSS_PAPER, c=0.023, Z=Z)
    for k in ("pdf_qr", "pdf_eps", "pdf_ens"):
        Hd = OM.hellinger(sur[k], ref[k])
        parity_log("surrogate 512-point mixture vs member quadrature, %s Hellinger" % k, Hd, 0.02)
        assert Hd <= 0.02, (k, Hd)
    S.close()


def test_surrogate_gain_over_nearest_member(E):
    """Train on the even-indexed members, evaluate at the held-out odd ones:
    the interpolant must beat taking the nearest simulated member (and is
    reported against linear interpolation in lambda)."""
    nq, nt = 16, 32
    h = E.hist_spec(qr_bins=nq, tail_bins=nt)
    lams = np.linspace(-3.0, 3.0, 17)
    counts = I.synthetic_member_counts(lams, nq, nt, 2_000_000, seed=4)
    P = OMLP.targets(counts, nq, nt)
    ev, od = np.arange(0, 17, 2), np.arange(1, 17, 2)
    S, _, _ = trained(E, lams[ev], counts[ev], h, steps=1500, seed=5)
    q = S.density(lams[od], h)
    hs, hn, hl = [], [], []
    for j, i in enumerate(od):
        hs.append(np.mean(hellinger_kinds(q[j], P[i], nq, nt)))
        hn.append(np.mean(hellinger_kinds(P[i - 1], P[i], nq, nt)))
        hl.append(np.mean(hellinger_kinds(0.5 * (P[i - 1] + P[i + 1]), P[i], nq, nt)))
    hs, hn, hl = np.mean(hs), np.mean(hn), np.mean(hl)
    print("held-out Hellinger: surrogate %.4f nearest member %.4f linear in lambda %.4f" % (hs, hn, hl))
    assert hs < hn
    S.close()
