"""C-ABI boundary checks that need no GPU: the library loads, exports every
symbol include/ens.h declares, rejects invalid members on the host, and the
binding refuses to run without a GPU (no CPU fallback)."""
import ctypes
import re

import pytest

import paper_2506_23712_gb300.ens as E
from paper_2506_23712_gb300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    return E.lib()


def header_symbols():
    with open(B.os.path.join(B.ROOT, "include", "ens.h")) as f:
        text = f.read()
    return set(re.findall(r"^(?:[a-z_ ]+\*?\s*)?\*?(ens_[a-z_]+)\s*\(", text, re.M)) | set(
        re.findall(r"\b(ens_[a-z_]+)\s*\((?:const )?ens_", text))


def test_every_declared_symbol_is_exported(lib):
    decl = header_symbols()
    assert {"ens_create", "ens_step", "ens_gradient_stats", "ens_mixture"} <= decl
    for name in decl:
        assert hasattr(lib, name), name
    assert decl == {n for n, _, _ in E.SIGNATURES}


def test_status_strings(lib):
    for code in range(8):
        assert lib.ens_status_string(code)
    assert lib.ens_status_string(0) == b"ok"


def test_query_validates_on_host(lib):
    h = E.hist_spec()
    ok = E.Member(N=32, nu=0.02, k_lo=1, k_hi=2).c()
    assert E.ens_query([ok], h) > 0
    with pytest.raises(E.EnsError) as e:
        E.ens_query([E.Member(N=30, nu=0.02).c()], h)
    assert e.value.status == 7
    with pytest.raises(E.EnsError) as e:   # band beyond the dealiased set (kc = 10 at N = 32)
        E.ens_query([E.Member(N=32, nu=0.02, k_lo=9, k_hi=11).c()], h)
    assert e.value.status == 1
    with pytest.raises(E.EnsError):
        E.ens_query([E.Member(N=32, nu=-1.0).c()], h)
    # degenerate forcing bands: no wave vector at all, only k = 0, or only
    # |k|^2 = 7 (not a sum of three squares): the forcing amplitude would be
    # undefined (E_B = 0)
    for lo, hi in ((2.5, 2.6), (0.0, 0.5), (7 ** 0.5, 7 ** 0.5)):
        with pytest.raises(E.EnsError) as e:
            E.ens_query([E.Member(N=32, nu=0.02, k_lo=lo, k_hi=hi).c()], h)
        assert e.value.status == 1, (lo, hi)
    assert E.ens_query([E.Member(N=32, nu=0.02, k_lo=6 ** 0.5, k_hi=6 ** 0.5).c()], h) > 0   # (1, 1, 2)
    with pytest.raises(E.EnsError):        # no members
        E.ens_query([], h)
    with pytest.raises(E.EnsError):        # mixed RK orders
        E.ens_query([E.Member(N=32, nu=0.02, rk_order=2).c(), E.Member(N=32, nu=0.02, rk_order=3).c()], h)
    # workspace grows with the member count and with N
    a = E.ens_query([ok], h)
    b = E.ens_query([ok, ok], h)
    c = E.ens_query([E.Member(N=64, nu=0.02).c()], h)
    assert b > a and c > a


def test_counts_len(lib):
    assert E.ens_counts_len(E.hist_spec(qr_bins=64, tail_bins=256)) == 64 * 64 + 512 + 8
    # gradient-component histograms append 2 x grad_bins + 4 counters
    assert E.ens_counts_len(E.hist_spec(qr_bins=64, tail_bins=256, grad_bins=100)) == 64 * 64 + 512 + 8 + 204


def test_binding_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        E.Ensemble([E.Member(N=32, nu=0.02)])


def test_workspace_too_small_is_enomem_before_any_device_call(lib, capfd):
    """ens_create with a caller-owned workspace one byte short of ens_query's
    size returns ENS_ENOMEM and no context, checked on the host before any
    CUDA call (the pointer is never dereferenced)."""
    h = E.hist_spec()
    ms = [E.Member(N=32, nu=0.02, k_lo=1, k_hi=2).c(), E.Member(N=64, nu=0.02, k_lo=1, k_hi=2).c()]
    need = E.ens_query(ms, h)
    arr = (E.MemberDesc * len(ms))(*ms)
    ctx = ctypes.c_void_p(12345)
    st = lib.ens_create(arr, len(ms), ctypes.byref(h), ctypes.c_void_p(1 << 20), need - 1, None, ctypes.byref(ctx))
    assert st == 2 and not ctx.value
    assert "workspace" in capfd.readouterr().err


def test_noalloc_limits_match_header(lib):
    with open(B.os.path.join(B.ROOT, "include", "ens.h")) as f:
        text = f.read()
    for name in ("ENS_NOALLOC_MAX_MEMBERS", "ENS_NOALLOC_MAX_COUNTS", "ENS_NMOM"):
        m = re.search(r"#define\s+%s\s+(\d+)" % name, text)
        assert m and int(m.group(1)) == getattr(E, name), name
