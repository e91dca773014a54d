"""Thin Python binding of libens (include/ens.h).

Argument marshalling only: every computation runs in the CUDA library.
PyTorch provides the device workspace (``torch.empty`` on the GPU) and the
CUDA stream (the current torch stream).  There is no CPU fallback: if the
library is missing or no GPU is present the calls fail loudly.

The module exposes the C entry points under their C names (``ens_create``,
``ens_step``, ``ens_gradient_stats``, ``ens_mixture``, ...) plus
:class:`Ensemble`, a small owner object that keeps the workspace alive.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libens.so")

ENS_NMOM = 48
ENS_NCOUNTERS = 8
STATUS = {0: "ENS_OK", 1: "ENS_EINVAL", 2: "ENS_ENOMEM", 3: "ENS_ECUDA", 4: "ENS_ENONFINITE",
          5: "ENS_ETIMEOUT", 6: "ENS_ESTATE", 7: "ENS_EUNSUPPORTED"}
W_GAUSS_PAPER, W_GAUSS, W_USER, W_TRUNC_GAUSS = 0, 1, 2, 3


class EnsError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))


class MemberDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("rk_order", ctypes.c_int), ("nu", ctypes.c_double),
                ("lam", ctypes.c_double), ("eps_bar", ctypes.c_double), ("k_lo", ctypes.c_double),
                ("k_hi", ctypes.c_double), ("dt", ctypes.c_double), ("cfl", ctypes.c_double),
                ("dt_max", ctypes.c_double), ("seed", ctypes.c_uint64), ("init_energy", ctypes.c_double)]


class HistSpec(ctypes.Structure):
    _fields_ = [("qr_bins", ctypes.c_int), ("q_lim", ctypes.c_double), ("r_lim", ctypes.c_double),
                ("tail_bins", ctypes.c_int), ("tail_lo", ctypes.c_double), ("tail_hi", ctypes.c_double),
                ("eps_norm", ctypes.c_double), ("nu_norm", ctypes.c_double), ("grad_bins", ctypes.c_int),
                ("grad_lim", ctypes.c_double)]


class Diag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("t", "dt", "E", "diss", "EB", "P", "umax", "Rlambda", "kmeta")] + \
               [("steps", ctypes.c_int64), ("flags", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class WeightSpec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("c", ctypes.c_double), ("Z", ctypes.c_double), ("mu", ctypes.c_double),
                ("sigma", ctypes.c_double), ("user", ctypes.POINTER(ctypes.c_double)), ("renormalize", ctypes.c_int)]


class MixtureOut(ctypes.Structure):
    _fields_ = [("weights", ctypes.POINTER(ctypes.c_double)), ("covered", ctypes.c_double),
                ("pdf_qr", ctypes.POINTER(ctypes.c_double)), ("pdf_eps", ctypes.POINTER(ctypes.c_double)),
                ("pdf_ens", ctypes.POINTER(ctypes.c_double)), ("moments", ctypes.POINTER(ctypes.c_double)),
                ("ratios", ctypes.c_double * 5), ("pdf_long", ctypes.POINTER(ctypes.c_double)),
                ("pdf_trans", ctypes.POINTER(ctypes.c_double))]


ENS_ZETA_QUADRATIC, ENS_ZETA_LOGPOISSON, ENS_ZETA_RATIONAL = 0, 1, 2
ENS_LAMBDA_GRID, ENS_LAMBDA_GRID_LO, ENS_LAMBDA_GRID_HI = 65536, -30.0, 30.0


class ZetaSpec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("c", ctypes.c_double), ("beta", ctypes.c_double), ("C0", ctypes.c_double)]


ENS_MAX_GROUPS = 8


class GroupTuning(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
                ("z_variant", ctypes.c_int), ("z_ctas_per_sm", ctypes.c_int), ("plan_x", ctypes.c_int),
                ("fx_split", ctypes.c_int)]


class Tuning(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_int), ("parallel_groups", ctypes.c_int), ("persistent", ctypes.c_int),
                ("group", GroupTuning * ENS_MAX_GROUPS), ("ms_per_step", ctypes.c_double),
                ("trials", ctypes.c_int)]


# every symbol declared in include/ens.h: (name, restype, argtypes)
_P = ctypes.POINTER
_vp, _i, _d, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
SIGNATURES = [
    ("ens_query", _i, [_P(MemberDesc), _i, _P(HistSpec), _P(_sz)]),
    ("ens_create", _i, [_P(MemberDesc), _i, _P(HistSpec), _vp, _sz, _vp, _P(_vp)]),
    ("ens_destroy", _i, [_vp]),
    ("ens_last_error", ctypes.c_char_p, [_vp]),
    ("ens_status_string", ctypes.c_char_p, [_i]),
    ("ens_step", _i, [_vp, _i]),
    ("ens_step_nograph", _i, [_vp, _i]),
    ("ens_step_sequential", _i, [_vp, _i]),
    ("ens_step_host", _i, [_vp, _vp, _vp, _sz, _i]),
    ("ens_get_tuning", _i, [_vp, _P(Tuning)]),
    ("ens_set_tuning", _i, [_vp, _P(Tuning)]),
    ("ens_autotune", _i, [_vp, _i, _P(Tuning)]),
    ("ens_gradient_stats", _i, [_vp, _i]),
    ("ens_get_stats", _i, [_vp, _vp, _vp]),
    ("ens_counts_len", _i, [_P(HistSpec)]),
    ("ens_mixture", _i, [_vp, _P(WeightSpec), _P(MixtureOut)]),
    ("ens_mixture_host", _i, [_i, _vp, _vp, _vp, _P(HistSpec), _P(WeightSpec), _P(MixtureOut), _vp]),
    ("ens_mixture_host_noalloc", _i, [_i, _vp, _vp, _vp, _P(HistSpec), _P(WeightSpec), _P(MixtureOut), _vp]),
    ("ens_lambda_pdf", _i, [_P(ZetaSpec), _d, _vp, _vp]),
    ("ens_lambda_weights", _i, [_P(ZetaSpec), _d, _i, _vp, _vp, _P(_d), _vp]),
    ("ens_nelkin_exponents", _i, [_P(ZetaSpec), _i, _vp, _vp]),
    ("ens_ratio_exponents", _i, [_P(ZetaSpec), _vp]),
    ("ens_scale_gap", _i, [_i, _vp, _vp, _d, _P(_d), _P(_d)]),
    ("ens_set_timestep", _i, [_vp, _i, _d, _d, _d]),
    ("ens_save", _i, [_vp, ctypes.c_char_p]),
    ("ens_load", _i, [_vp, ctypes.c_char_p]),
    ("ens_get_field", _i, [_vp, _i, _vp]),
    ("ens_set_field", _i, [_vp, _i, _vp]),
    ("ens_state_bytes", _sz, [_vp]),
    ("ens_get_state", _i, [_vp, _vp, _sz]),
    ("ens_set_state", _i, [_vp, _vp, _sz]),
    ("ens_get_velocity", _i, [_vp, _i, _vp]),
    ("ens_set_velocity", _i, [_vp, _i, _vp]),
    ("ens_rhs", _i, [_vp, _i, _vp]),
    ("ens_diagnostics", _i, [_vp, _P(Diag)]),
    ("ens_synchronize", _i, [_vp]),
    ("ens_test_skip_copy", _i, [_vp, _i, _i]),
    ("ens_members", _i, [_vp]),
    ("ens_member_n", _i, [_vp, _i]),
    ("ens_run_pass", _i, [_vp, _i, _i]),
    ("ens_kernels_per_step", _i, [_vp]),
    ("ens_pass_bytes", _d, [_vp, _i, _i]),
    ("ens_surrogate_create", _i, [ctypes.c_uint64, _vp, _P(_vp)]),
    ("ens_surrogate_destroy", _i, [_vp]),
    ("ens_surrogate_param_count", _sz, []),
    ("ens_surrogate_get_params", _i, [_vp, _vp]),
    ("ens_surrogate_set_params", _i, [_vp, _vp]),
    ("ens_surrogate_loss_grad", _i, [_vp, _i, _vp, _vp, _P(HistSpec), _P(_d), _vp]),
    ("ens_surrogate_train", _i, [_vp, _i, _vp, _vp, _P(HistSpec), _i, _d, _P(_d)]),
    ("ens_surrogate_density", _i, [_vp, _i, _vp, _P(HistSpec), _vp]),
    ("ens_surrogate_mixture", _i, [_vp, _P(HistSpec), _P(WeightSpec), _d, _d, _i, _P(MixtureOut)]),
    ("ens_surrogate_time_gemm", _i, [_vp, ctypes.c_longlong, _i, _P(_d)]),
    ("ens_surrogate_logits", _i, [_vp, _i, _vp, _P(HistSpec), _i, _vp]),
    ("ens_surrogate_time_infer", _i, [_vp, _P(HistSpec), _i, _i, _P(_d)]),
    ("ens_tc_gemm_check", _i, [_vp, _vp, _vp, _i, _i, _i, _i]),
    ("ens_bin_check", _i, [_vp, _i, _vp, _i, _vp]),
]

_lib = None


def lib():
    """Load libens.so (built by ``__graft_entry__.build()``); no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libens.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status, ctx=None):
    if status != 0:
        msg = lib().ens_last_error(ctx).decode() if ctx else ""
        raise EnsError(status, msg)


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
# C entry points under their own names (marshalling only)
# ---------------------------------------------------------------------------
def ens_query(members: Sequence[MemberDesc], hist: HistSpec) -> int:
    arr = (MemberDesc * len(members))(*members)
    out = ctypes.c_size_t()
    _check(lib().ens_query(arr, len(members), ctypes.byref(hist), ctypes.byref(out)))
    return out.value


def ens_create(members, hist, workspace_ptr, workspace_bytes, stream_ptr):
    arr = (MemberDesc * len(members))(*members)
    ctx = ctypes.c_void_p()
    _check(lib().ens_create(arr, len(members), ctypes.byref(hist), ctypes.c_void_p(workspace_ptr),
                            workspace_bytes, stream_ptr, ctypes.byref(ctx)))
    return ctx


def ens_destroy(ctx):
    _check(lib().ens_destroy(ctx))


def ens_step(ctx, nsteps=1):
    _check(lib().ens_step(ctx, nsteps), ctx)


def ens_step_nograph(ctx, nsteps=1):
    _check(lib().ens_step_nograph(ctx, nsteps), ctx)


def ens_step_sequential(ctx, nsteps=1):
    _check(lib().ens_step_sequential(ctx, nsteps), ctx)


_GROUP_KEYS = ("N", "tile_x", "tile_y", "z_variant", "z_ctas_per_sm", "plan_x", "fx_split")


def _tuning_dict(t: Tuning) -> dict:
    return {"parallel_groups": t.parallel_groups, "persistent": t.persistent,
            "groups": [{k: getattr(t.group[i], k) for k in _GROUP_KEYS} for i in range(t.groups)],
            "ms_per_step": t.ms_per_step, "trials": t.trials}


def ens_get_tuning(ctx) -> dict:
    t = Tuning()
    _check(lib().ens_get_tuning(ctx, ctypes.byref(t)), ctx)
    return _tuning_dict(t)


def ens_set_tuning(ctx, tuning: dict):
    t = Tuning()
    t.groups = len(tuning["groups"])
    t.parallel_groups = int(tuning["parallel_groups"])
    t.persistent = int(tuning.get("persistent", 0))
    for i, g in enumerate(tuning["groups"]):
        for k in _GROUP_KEYS:
            setattr(t.group[i], k, int(g[k]))
    _check(lib().ens_set_tuning(ctx, ctypes.byref(t)), ctx)


def ens_autotune(ctx, steps=3) -> dict:
    t = Tuning()
    _check(lib().ens_autotune(ctx, steps, ctypes.byref(t)), ctx)
    return _tuning_dict(t)


def ens_gradient_stats(ctx, accumulate=True):
    _check(lib().ens_gradient_stats(ctx, int(bool(accumulate))), ctx)


def ens_counts_len(hist: HistSpec) -> int:
    return lib().ens_counts_len(ctypes.byref(hist))


def ens_get_stats(ctx, n, counts_len):
    counts = np.zeros((n, counts_len), dtype=np.uint64)
    moments = np.zeros((n, ENS_NMOM), dtype=np.float64)
    _check(lib().ens_get_stats(ctx, _ptr(counts), _ptr(moments)), ctx)
    return counts, moments


def _weight_spec(kind, c=0.023, Z=1.0, mu=0.0, sigma=1.0, user=None, renormalize=True):
    ws = WeightSpec(kind, c, Z, mu, sigma, None, int(bool(renormalize)))
    keep = None
    if user is not None:
        keep = np.ascontiguousarray(user, dtype=np.float64)
        ws.user = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return ws, keep


def _mixture_out(n, hist):
    nq, nt = hist.qr_bins, hist.tail_bins
    bufs = {"weights": np.zeros(n), "pdf_qr": np.zeros(nq * nq), "pdf_eps": np.zeros(nt),
            "pdf_ens": np.zeros(nt), "moments": np.zeros(ENS_NMOM)}
    if hist.grad_bins > 0:
        bufs["pdf_long"] = np.zeros(hist.grad_bins)
        bufs["pdf_trans"] = np.zeros(hist.grad_bins)
    out = MixtureOut()
    for k, v in bufs.items():
        setattr(out, k, v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out, bufs


def _mixture_result(out, bufs, hist):
    nq = hist.qr_bins
    return {"weights": bufs["weights"], "covered": out.covered, "pdf_qr": bufs["pdf_qr"].reshape(nq, nq),
            "pdf_eps": bufs["pdf_eps"], "pdf_ens": bufs["pdf_ens"], "moments": bufs["moments"],
            "pdf_long": bufs.get("pdf_long"), "pdf_trans": bufs.get("pdf_trans"),
            "ratios": dict(zip(("S_long", "F_long", "F_trans", "H_long", "H_trans"), list(out.ratios)))}


def ens_mixture(ctx, n, hist, **weights):
    ws, keep = _weight_spec(**weights)
    out, bufs = _mixture_out(n, hist)
    _check(lib().ens_mixture(ctx, ctypes.byref(ws), ctypes.byref(out)), ctx)
    return _mixture_result(out, bufs, hist)


def _host_stats_arrays(lambdas, counts, moments, hist, weights):
    """The host inputs of the mixture as contiguous arrays, their shapes
    checked against the member count and the histogram layout (the C side
    reads n * counts_len counts, n * ENS_NMOM moments and n user weights)."""
    lam = np.ascontiguousarray(lambdas, dtype=np.float64).ravel()
    counts = np.ascontiguousarray(counts, dtype=np.uint64)
    moments = np.ascontiguousarray(moments, dtype=np.float64)
    n = lam.size
    L = ens_counts_len(hist)
    if counts.shape != (n, L):
        raise ValueError("counts has shape %s, expected (%d, %d)" % (counts.shape, n, L))
    if moments.shape != (n, ENS_NMOM):
        raise ValueError("moments has shape %s, expected (%d, %d)" % (moments.shape, n, ENS_NMOM))
    user = weights.get("user")
    if user is not None and np.asarray(user).size != n:
        raise ValueError("%d user weights for %d members" % (np.asarray(user).size, n))
    return lam, counts, moments, n


def ens_mixture_host(lambdas, counts, moments, hist, stream_ptr=None, **weights):
    lam, counts, moments, n = _host_stats_arrays(lambdas, counts, moments, hist, weights)
    ws, keep = _weight_spec(**weights)
    out, bufs = _mixture_out(n, hist)
    if stream_ptr is None:
        stream_ptr = _stream_ptr()
    _check(lib().ens_mixture_host(n, _ptr(lam), _ptr(counts), _ptr(moments), ctypes.byref(hist),
                                  ctypes.byref(ws), ctypes.byref(out), stream_ptr))
    return _mixture_result(out, bufs, hist)


ENS_NOALLOC_MAX_MEMBERS = 64
ENS_NOALLOC_MAX_COUNTS = 8192


def ens_mixture_host_noalloc(lambdas, counts, moments, hist, stream_ptr=None, **weights):
    """ens_mixture_host without device allocation (fixed library scratch);
    for callers that cannot allocate device memory.  Raises EnsError with
    ENS_EINVAL beyond ENS_NOALLOC_MAX_MEMBERS members or
    ENS_NOALLOC_MAX_COUNTS counts per member."""
    lam, counts, moments, n = _host_stats_arrays(lambdas, counts, moments, hist, weights)
    ws, keep = _weight_spec(**weights)
    out, bufs = _mixture_out(n, hist)
    if stream_ptr is None:
        stream_ptr = _stream_ptr()
    _check(lib().ens_mixture_host_noalloc(n, _ptr(lam), _ptr(counts), _ptr(moments), ctypes.byref(hist),
                                          ctypes.byref(ws), ctypes.byref(out), stream_ptr))
    return _mixture_result(out, bufs, hist)


def zeta_spec(kind="quadratic", c=0.023, beta=None, C0=2.0) -> ZetaSpec:
    """zeta_p family: 'quadratic' (c), 'logpoisson' (beta, default 2/3; C0)
    or 'rational' (beta, default 0.05)."""
    z = ZetaSpec()
    z.kind = {"quadratic": ENS_ZETA_QUADRATIC, "logpoisson": ENS_ZETA_LOGPOISSON,
              "rational": ENS_ZETA_RATIONAL}[kind]
    if beta is None:
        beta = 0.05 if kind == "rational" else 2.0 / 3.0
    z.c, z.beta, z.C0 = c, beta, C0
    return z


def lambda_grid() -> np.ndarray:
    return ENS_LAMBDA_GRID_LO + np.arange(ENS_LAMBDA_GRID) * (
        (ENS_LAMBDA_GRID_HI - ENS_LAMBDA_GRID_LO) / ENS_LAMBDA_GRID)


def ens_lambda_pdf(zeta: ZetaSpec, Z: float, stream_ptr=None) -> np.ndarray:
    out = np.empty(ENS_LAMBDA_GRID, dtype=np.float64)
    if stream_ptr is None:
        stream_ptr = _stream_ptr()
    _check(lib().ens_lambda_pdf(ctypes.byref(zeta), Z, _ptr(out), stream_ptr))
    return out


def ens_lambda_weights(zeta: ZetaSpec, Z: float, lambdas, stream_ptr=None):
    """(weights, covered) of the members for the lambda law of `zeta` at Z."""
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    w = np.empty(lam.size, dtype=np.float64)
    cov = ctypes.c_double()
    if stream_ptr is None:
        stream_ptr = _stream_ptr()
    _check(lib().ens_lambda_weights(ctypes.byref(zeta), Z, lam.size, _ptr(lam), _ptr(w), ctypes.byref(cov),
                                    stream_ptr))
    return w, cov.value


def ens_nelkin_exponents(zeta: ZetaSpec, m) -> np.ndarray:
    mm = np.ascontiguousarray(m, dtype=np.float64)
    rho = np.empty(mm.size, dtype=np.float64)
    _check(lib().ens_nelkin_exponents(ctypes.byref(zeta), mm.size, _ptr(mm), _ptr(rho)))
    return rho


def ens_ratio_exponents(zeta: ZetaSpec):
    out = np.empty(3, dtype=np.float64)
    _check(lib().ens_ratio_exponents(ctypes.byref(zeta), _ptr(out)))
    return tuple(out)


def ens_scale_gap(lambdas, rlambda, R_ref):
    """(Z, R0) for a target R_lambda from the members' R_lambda."""
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    r = np.ascontiguousarray(rlambda, dtype=np.float64)
    if r.size != lam.size:
        raise ValueError("one R_lambda per member")
    Z, R0 = ctypes.c_double(), ctypes.c_double()
    _check(lib().ens_scale_gap(lam.size, _ptr(lam), _ptr(r), R_ref, ctypes.byref(Z), ctypes.byref(R0)))
    return Z.value, R0.value


def ens_set_timestep(ctx, member: int, dt: float, cfl: float, dt_max: float):
    _check(lib().ens_set_timestep(ctx, member, dt, cfl, dt_max), ctx)


def ens_save(ctx, path: str):
    _check(lib().ens_save(ctx, path.encode()), ctx)


def ens_load(ctx, path: str):
    _check(lib().ens_load(ctx, path.encode()), ctx)


def _full_shape(N):
    return (3, N, N, N // 2 + 1)


def ens_get_field(ctx, member, N):
    out = np.zeros(_full_shape(N), dtype=np.complex128)
    _check(lib().ens_get_field(ctx, member, _ptr(out)), ctx)
    return out


def ens_set_field(ctx, member, field_):
    a = np.ascontiguousarray(field_, dtype=np.complex128)
    _check(lib().ens_set_field(ctx, member, _ptr(a)), ctx)


def ens_get_velocity(ctx, member, N):
    out = np.zeros((3, N, N, N), dtype=np.float64)
    _check(lib().ens_get_velocity(ctx, member, _ptr(out)), ctx)
    return out


def ens_set_velocity(ctx, member, u):
    a = np.ascontiguousarray(u, dtype=np.float64)
    _check(lib().ens_set_velocity(ctx, member, _ptr(a)), ctx)


def ens_rhs(ctx, member, N):
    out = np.zeros(_full_shape(N), dtype=np.complex128)
    _check(lib().ens_rhs(ctx, member, _ptr(out)), ctx)
    return out


def ens_state_bytes(ctx) -> int:
    return lib().ens_state_bytes(ctx)


def ens_get_state(ctx, host_ptr, nbytes):
    _check(lib().ens_get_state(ctx, ctypes.c_void_p(host_ptr), nbytes), ctx)


def ens_set_state(ctx, host_ptr, nbytes):
    _check(lib().ens_set_state(ctx, ctypes.c_void_p(host_ptr), nbytes), ctx)


def ens_step_host(ctx, host_in_ptr, host_out_ptr, nbytes, chunk=0):
    _check(lib().ens_step_host(ctx, ctypes.c_void_p(host_in_ptr), ctypes.c_void_p(host_out_ptr), nbytes, chunk), ctx)


DIAG_KEYS = ("t", "dt", "E", "diss", "EB", "P", "umax", "Rlambda", "kmeta", "steps", "flags")


def ens_diagnostics(ctx, n, raise_on_flag=True):
    arr = (Diag * n)()
    st = lib().ens_diagnostics(ctx, arr)
    if st not in (0, 4, 5, 6) or (raise_on_flag and st != 0):
        _check(st, ctx)
    return [{k: getattr(d, k) for k in DIAG_KEYS} for d in arr], st


def ens_synchronize(ctx):
    _check(lib().ens_synchronize(ctx), ctx)


def ens_test_skip_copy(ctx, member, wait_polls):
    _check(lib().ens_test_skip_copy(ctx, member, wait_polls), ctx)


def ens_run_pass(ctx, pass_id, stage=0):
    _check(lib().ens_run_pass(ctx, pass_id, stage), ctx)


def ens_pass_bytes(ctx, pass_id, stage=0) -> float:
    return lib().ens_pass_bytes(ctx, pass_id, stage)


def ens_kernels_per_step(ctx) -> int:
    return lib().ens_kernels_per_step(ctx)


# ---------------------------------------------------------------------------
# owner object
# ---------------------------------------------------------------------------
@dataclass
class Member:
    """One ensemble member (mirrors ens_member_desc)."""
    N: int
    nu: float
    lam: float = 0.0
    eps_bar: float = 0.1
    k_lo: float = 1.0
    k_hi: float = 2.0
    dt: float = 0.01
    cfl: float = 0.2
    dt_max: float = 0.0
    rk_order: int = 3
    seed: int = 0
    init_energy: float = 0.5

    def c(self) -> MemberDesc:
        return MemberDesc(self.N, self.rk_order, self.nu, self.lam, self.eps_bar, self.k_lo, self.k_hi, self.dt,
                          self.cfl, self.dt_max, self.seed, self.init_energy)


def hist_spec(qr_bins=64, q_lim=10.0, r_lim=10.0, tail_bins=256, tail_lo=-8.0, tail_hi=8.0, eps_norm=0.1,
              nu_norm=0.01, grad_bins=0, grad_lim=40.0) -> HistSpec:
    return HistSpec(qr_bins, q_lim, r_lim, tail_bins, tail_lo, tail_hi, eps_norm, nu_norm, grad_bins, grad_lim)


class Ensemble:
    """An ensemble on the current CUDA device.  Torch allocates the device
    workspace and supplies the stream; libens does all the work."""

    def __init__(self, members: Sequence[Member], hist: Optional[HistSpec] = None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libens needs a CUDA GPU; no CPU fallback exists")
        self.members = list(members)
        self.hist = hist if hist is not None else hist_spec(nu_norm=self.members[0].nu,
                                                             eps_norm=self.members[0].eps_bar)
        descs = [m.c() for m in self.members]
        nbytes = ens_query(descs, self.hist)
        self._ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = ens_create(descs, self.hist, self._ws.data_ptr(), nbytes, _stream_ptr(self._stream))
        self.counts_len = ens_counts_len(self.hist)

    @property
    def n(self):
        return len(self.members)

    def step(self, nsteps=1, graph=True):
        (ens_step if graph else ens_step_nograph)(self.ctx, nsteps)

    def save(self, path: str):
        ens_save(self.ctx, path)

    def set_timestep(self, member: int, dt: float, cfl: float, dt_max: float):
        ens_set_timestep(self.ctx, member, dt, cfl, dt_max)

    def load(self, path: str):
        ens_load(self.ctx, path)

    def tuning(self) -> dict:
        return ens_get_tuning(self.ctx)

    def set_tuning(self, tuning: dict):
        ens_set_tuning(self.ctx, tuning)

    def tuning_key(self) -> str:
        """Cache key of a tuning: device name, RK order and the member count
        per grid size."""
        import torch
        sizes = {}
        for m in self.members:
            sizes[m.N] = sizes.get(m.N, 0) + 1
        return "%s|rk%d|%s" % (torch.cuda.get_device_name(), self.members[0].rk_order,
                                ",".join("%dx%d" % (c, n) for n, c in sorted(sizes.items())))

    def autotune(self, steps=3, cache: Optional[str] = None) -> dict:
        """Install the fastest pass variants for this ensemble.  With a cache
        path (a JSON file), a tuning stored under this ensemble's key is
        installed without timing anything; otherwise the library times the
        variants (ens_autotune) and the result is stored there."""
        import json
        import os
        key = self.tuning_key()
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
            if key in table:
                self.set_tuning(table[key])
                return dict(table[key], cached=True)
        t = ens_autotune(self.ctx, steps)
        if cache:
            table[key] = t
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return dict(t, cached=False)

    def gradient_stats(self, accumulate=True):
        ens_gradient_stats(self.ctx, accumulate)

    def stats(self):
        return ens_get_stats(self.ctx, self.n, self.counts_len)

    def mixture(self, **weights):
        return ens_mixture(self.ctx, self.n, self.hist, **weights)

    def field(self, i):
        return ens_get_field(self.ctx, i, self.members[i].N)

    def set_field(self, i, f):
        ens_set_field(self.ctx, i, f)

    def velocity(self, i):
        return ens_get_velocity(self.ctx, i, self.members[i].N)

    def set_velocity(self, i, u):
        ens_set_velocity(self.ctx, i, u)

    def rhs(self, i):
        return ens_rhs(self.ctx, i, self.members[i].N)

    def diagnostics(self, raise_on_flag=True):
        return ens_diagnostics(self.ctx, self.n, raise_on_flag)[0]

    def synchronize(self):
        ens_synchronize(self.ctx)

    def state_bytes(self):
        return ens_state_bytes(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            ens_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# learned lambda interpolant (surrogate)
# ---------------------------------------------------------------------------
def ens_bin_check(ctx, axis, values):
    """The statistics pass's bin rule on FP32 values in an axis's units
    (0 Q/q0, 1 R/q0^1.5, 2 log10 tail, 3 A_ij/sqrt(q0)), on the device."""
    x = np.ascontiguousarray(values, dtype=np.float32)
    out = np.empty(x.size, dtype=np.int32)
    _check(lib().ens_bin_check(ctx, axis, _ptr(x), x.size, _ptr(out)))
    return out


def ens_tc_gemm_check(A_bf16_bits, B_bf16_bits, ksplit=1):
    """C = A B^T on the tensor cores; A [M][K], B [N][K] as uint16 BF16 bits."""
    A = np.ascontiguousarray(A_bf16_bits, dtype=np.uint16)
    B = np.ascontiguousarray(B_bf16_bits, dtype=np.uint16)
    M, K = A.shape
    N = B.shape[0]
    C = np.zeros((M, N), dtype=np.float32)
    _check(lib().ens_tc_gemm_check(_ptr(A), _ptr(B), _ptr(C), M, N, K, ksplit))
    return C


class Surrogate:
    """Owner of an ens_surrogate (MLP over (bin, lambda) on the tensor cores)."""

    def __init__(self, seed=0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libens needs a CUDA GPU; no CPU fallback exists")
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(lib().ens_surrogate_create(seed, _stream_ptr(self._stream), ctypes.byref(h)))
        self.h = h
        self.nparam = lib().ens_surrogate_param_count()

    def params(self):
        out = np.zeros(self.nparam, dtype=np.float32)
        _check(lib().ens_surrogate_get_params(self.h, _ptr(out)))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparam
        _check(lib().ens_surrogate_set_params(self.h, _ptr(p)))

    def loss_grad(self, lambdas, counts, hist):
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        counts = np.ascontiguousarray(counts, dtype=np.uint64)
        g = np.zeros(self.nparam, dtype=np.float32)
        loss = ctypes.c_double()
        _check(lib().ens_surrogate_loss_grad(self.h, lam.size, _ptr(lam), _ptr(counts), ctypes.byref(hist),
                                             ctypes.byref(loss), _ptr(g)))
        return loss.value, g

    def train(self, lambdas, counts, hist, steps, lr=1e-3):
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        counts = np.ascontiguousarray(counts, dtype=np.uint64)
        loss = ctypes.c_double()
        _check(lib().ens_surrogate_train(self.h, lam.size, _ptr(lam), _ptr(counts), ctypes.byref(hist), steps, lr,
                                         ctypes.byref(loss)))
        return loss.value

    def density(self, lambdas, hist):
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        per = hist.qr_bins ** 2 + 2 * hist.tail_bins
        out = np.zeros((lam.size, per), dtype=np.float64)
        _check(lib().ens_surrogate_density(self.h, lam.size, _ptr(lam), ctypes.byref(hist), _ptr(out)))
        return out

    def logits(self, lambdas, hist, fused=True):
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        per = hist.qr_bins ** 2 + 2 * hist.tail_bins
        out = np.zeros((lam.size, per), dtype=np.float32)
        _check(lib().ens_surrogate_logits(self.h, lam.size, _ptr(lam), ctypes.byref(hist), int(bool(fused)),
                                          _ptr(out)))
        return out

    def time_infer(self, hist, nquad=512, iters=5):
        ms = ctypes.c_double()
        _check(lib().ens_surrogate_time_infer(self.h, ctypes.byref(hist), nquad, iters, ctypes.byref(ms)))
        return ms.value

    def time_gemm(self, rows, iters=10):
        ms = ctypes.c_double()
        _check(lib().ens_surrogate_time_gemm(self.h, rows, iters, ctypes.byref(ms)))
        return ms.value

    def mixture(self, hist, lam_lo, lam_hi, nquad=512, **weights):
        ws, keep = _weight_spec(**weights)
        out, bufs = _mixture_out(1, hist)
        _check(lib().ens_surrogate_mixture(self.h, ctypes.byref(hist), ctypes.byref(ws), lam_lo, lam_hi, nquad,
                                           ctypes.byref(out)))
        return _mixture_result(out, bufs, hist)

    def close(self):
        if getattr(self, "h", None):
            lib().ens_surrogate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
