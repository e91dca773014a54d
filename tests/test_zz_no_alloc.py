"""ens_mixture_host_noalloc: the mixture for callers that cannot allocate
device memory (their GPU memory is owned by another allocator or budgeted up
front).  It must give the same results as ens_mixture_host, call after call,
while keeping its inputs and outputs in the library's fixed scratch array.

Collected last on purpose: a failure here leaves every other test already run.
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


def synthetic_stats(n, hist, seed):
    """Seeded member statistics in the library's counts/moments layout."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    L = hist.qr_bins ** 2 + 2 * hist.tail_bins + 8      # the counters end the first block
    Lg = 2 * hist.grad_bins + 4 if hist.grad_bins > 0 else 0
    counts = rng.integers(0, 5000, size=(n, L + Lg)).astype(np.uint64)
    nbins = hist.qr_bins ** 2
    counts[:, L - 2] = counts[:, :nbins].sum(axis=1) + counts[:, L - 8]   # npoints
    moments = rng.standard_normal((n, 48)) ** 2 * 1e3
    lams = np.sort(rng.uniform(-5.1, 5.8, n))
    return lams, counts, moments


def compare(a, b):
    np.testing.assert_allclose(a["weights"], b["weights"], rtol=1e-13, atol=0)
    assert a["covered"] == pytest.approx(b["covered"], rel=1e-13)
    for k in ("pdf_qr", "pdf_eps", "pdf_ens", "moments"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-13, atol=1e-300)
    for k in ("pdf_long", "pdf_trans"):
        if b[k] is not None:
            np.testing.assert_allclose(a[k], b[k], rtol=1e-13, atol=1e-300)
    for k, v in b["ratios"].items():
        assert a["ratios"][k] == pytest.approx(v, rel=1e-13)


def test_noalloc_matches_allocating_mixture_twice(E):
    h = E.hist_spec(qr_bins=64, tail_bins=256)
    # two calls in a row with different inputs: the second must not see the first's data
    cases = [(48, 1, dict(kind=E.W_GAUSS_PAPER, c=0.023, Z=4.54)),
             (17, 2, dict(kind=E.W_TRUNC_GAUSS, c=0.023, Z=2.0))]
    for n, seed, w in cases:
        lams, counts, moments = synthetic_stats(n, h, seed)
        ref = E.ens_mixture_host(lams, counts, moments, h, **w)
        got = E.ens_mixture_host_noalloc(lams, counts, moments, h, **w)
        compare(got, ref)
        assert got["weights"].sum() == pytest.approx(1.0, rel=1e-12)


def test_noalloc_user_weights_and_limits(E):
    h = E.hist_spec(qr_bins=16, tail_bins=32)
    lams, counts, moments = synthetic_stats(5, h, 3)
    user = np.array([0.1, 0.2, 0.3, 0.25, 0.15])
    ref = E.ens_mixture_host(lams, counts, moments, h, kind=E.W_USER, user=user)
    got = E.ens_mixture_host_noalloc(lams, counts, moments, h, kind=E.W_USER, user=user)
    compare(got, ref)
    # beyond the fixed scratch: rejected on the host before any device work
    big_n = E.ENS_NOALLOC_MAX_MEMBERS + 1
    lams, counts, moments = synthetic_stats(big_n, h, 4)
    with pytest.raises(E.EnsError) as err:
        E.ens_mixture_host_noalloc(lams, counts, moments, h, kind=E.W_GAUSS, mu=0.0, sigma=1.5)
    assert err.value.status == 1
    wide = E.hist_spec(qr_bins=128, tail_bins=256)   # 128^2 + 512 + 8 counts > 8192
    lams, counts, moments = synthetic_stats(3, wide, 5)
    with pytest.raises(E.EnsError):
        E.ens_mixture_host_noalloc(lams, counts, moments, wide, kind=E.W_GAUSS, mu=0.0, sigma=1.5)


def test_noalloc_gradient_pdfs_and_no_device_allocation(E):
    """With gradient-component bins the counts carry the longitudinal and
    transverse blocks and their four counters: pdf_long and pdf_trans come
    back as from ens_mixture_host.  After a first call, two more calls of
    different sizes leave the device's free memory unchanged (an allocation
    would take at least one 2 MB page)."""
    hg = E.hist_spec(qr_bins=64, tail_bins=256, grad_bins=64, grad_lim=8.0)
    assert E.ens_counts_len(hg) <= E.ENS_NOALLOC_MAX_COUNTS
    lams, counts, moments = synthetic_stats(9, hg, 6)
    w = dict(kind=E.W_GAUSS, mu=-1.125, sigma=1.5)
    ref = E.ens_mixture_host(lams, counts, moments, hg, **w)
    got = E.ens_mixture_host_noalloc(lams, counts, moments, hg, **w)
    compare(got, ref)
    assert got["pdf_long"] is not None and np.any(got["pdf_long"] > 0) and np.any(got["pdf_trans"] > 0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    h2 = E.hist_spec(qr_bins=32, tail_bins=128)
    for (hh, n, seed) in ((hg, 40, 7), (h2, 3, 8)):
        lams, counts, moments = synthetic_stats(n, hh, seed)
        E.ens_mixture_host_noalloc(lams, counts, moments, hh, **w)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
