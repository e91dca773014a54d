"""The tcgen05 (tensor-core) BF16 GEMM against numpy on the same BF16 values.

Exact BF16 products accumulate in FP32 on both sides; only the summation
order differs, so the relative error is at the FP32 rounding level."""
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


def bf16_bits(x):
    """Round-to-nearest-even FP32 -> BF16 bit patterns, and their values."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    return r, (r.astype(np.uint32) << 16).view(np.float32)


@pytest.mark.parametrize("M,N,K,split", [(128, 64, 64, 1), (256, 128, 128, 1), (256, 256, 256, 1),
                                         (384, 256, 1024, 4), (128, 64, 2048, 8)])
def test_tc_gemm_matches_numpy(E, M, N, K, split):
    rng = np.random.Generator(np.random.Philox(key=M * 7 + N + K))
    a_bits, a = bf16_bits(rng.standard_normal((M, K)))
    b_bits, b = bf16_bits(rng.standard_normal((N, K)))
    C = E.ens_tc_gemm_check(a_bits, b_bits, split)
    ref = a.astype(np.float64) @ b.astype(np.float64).T
    err = np.abs(C - ref).max() / np.abs(ref).max()
    assert err < 1e-5, err
