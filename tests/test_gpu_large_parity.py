"""One-step parity of the RK step at the large grid sizes, in every pass
variant the autotuner can pick there, against the FP64 oracle.

* N = 128: members of the uneven-size batch (24 x 128^3 + 12 x 256^3 +
  4 x 384^3, nu per member for k_max eta >= 1.5, band [6, 8], IF-RK3,
  CFL 0.2), element by element on the whole field against the oracle run
  live; every combination of x-pass plan, x tile, split or fused last pass
  and z-pass variant.
* N = 256, 384, 512: the oracle step takes minutes there, so its result is
  stored (``tests/golden/one_step_<N>.npz``, written by
  ``tests/golden/make_oracle_goldens.py`` from ``oracle/`` alone) on a fixed
  sample of modes: every kept mode with max_i |k_i| <= 3, every forcing-band
  mode and 2048 seeded random kept modes, all three components.  Members:
  the central and the largest-lambda member of the 64 x 256^3 benchmark
  ensemble; the smallest- and largest-lambda 384^3 members of the uneven
  batch; the largest-lambda 512^3 member of the mixed-resolution ensemble
  (Sec. VI: high-lambda members on twice the resolution) and the 512^3
  reference-run shape (nu 0.0015, band [1, 2]).

Bounds (Sec. IV; the one-step tolerance of the FP32 path): relative L2 over
the compared modes <= 1e-5, the CFL time step and the energy within 1e-5,
the injected power exp(lambda) eps_bar within 1e-6.  The gradient statistics
of the stepped field (default variant) against the oracle's statistics of
its own stepped field: exact point count, 2% in every bin with more than
1000 counts, the totals within 0.1%.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import ens_inputs as I
import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
HIST = dict(qr_bins=64, q_lim=10.0, r_lim=10.0, tail_bins=256, tail_lo=-8.0, tail_hi=8.0, eps_norm=0.1)


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2506_23712_gb300 import build as B
    B.build()
    import paper_2506_23712_gb300.ens as ens
    return ens


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def lib_member(E, d):
    return E.Member(N=d["N"], nu=d["nu"], lam=d["lam"], eps_bar=d["eps_bar"], k_lo=d["k_lo"], k_hi=d["k_hi"],
                    dt=d["dt"], cfl=d["cfl"], dt_max=d["dt_max"], rk_order=d["rk_order"], seed=d["seed"],
                    init_energy=d["init_energy"])


def oracle_member(d):
    return O.Member(N=d["N"], nu=d["nu"], lam=d["lam"], eps_bar=d["eps_bar"], k_lo=d["k_lo"], k_hi=d["k_hi"],
                    dt=d["dt"], cfl=d["cfl"], dt_max=d["dt_max"], rk_order=d["rk_order"], seed=d["seed"],
                    init_energy=d["init_energy"])


def tunings(E, ens, N):
    """Every combination of the variants the autotuner searches at N (column
    tile of the x passes, x-pass FFT plan where a second one exists, fused,
    split or warp-group last pass, z-pass variant), the y tile and CTAs per SM
    at their defaults."""
    base = ens.tuning()
    plans = (0, 1) if N in (128, 256, 512) else (0,)
    zvars = (0, 1, 2) if N == 256 else (0, 1)
    splits = (0, 1, 2) if N == 256 else (0, 1)
    out = []
    for tx, plan, split, zv in itertools.product((16, 8), plans, splits, zvars):
        t = json.loads(json.dumps(base))
        t["groups"][0].update(tile_x=tx, plan_x=plan, fx_split=split, z_variant=zv)
        if zv == 2:
            t["groups"][0]["z_ctas_per_sm"] = 1
        out.append(t)
    return out


def check_stats(counts, ref, npts, parity_log, what):
    c, r = counts.astype(np.int64), ref.astype(np.int64)
    assert c[-2] == r[-2] == npts
    big = r > 1000
    assert big.sum() > 50
    dev = np.abs(c[big] - r[big]) / r[big]
    parity_log(what + " max bin deviation (bins > 1000 counts)", dev.max(), 0.02)
    assert dev.max() <= 0.02
    assert abs(int(c.sum()) - int(r.sum())) <= 1e-3 * r.sum()


# ---------------------------------------------------------------------------
# N = 128: whole field against the live oracle
# ---------------------------------------------------------------------------
def test_one_step_128_every_variant_matches_oracle(E, parity_log):
    ds = [d for d in I.uneven_batch() if d["N"] == 128]
    picks = [ds[0], ds[len(ds) // 2], ds[-1]]
    refs, rdiag = [], []
    for d in picks:
        om = oracle_member(d)
        uh = O.initial_field(om)
        st, od = O.step(om, uh, 1)
        assert st == 0
        refs.append(uh)
        rdiag.append(od)
    ms = [lib_member(E, d) for d in picks]
    probe = E.Ensemble(ms)
    variants = tunings(E, probe, 128)
    probe.close()
    worst = 0.0
    for t in variants:
        ens = E.Ensemble(ms)
        ens.set_tuning(t)
        ens.step(1)
        dg = ens.diagnostics()
        for i, d in enumerate(picks):
            err = rel(ens.field(i), refs[i])
            worst = max(worst, err)
            assert err < 1e-5, (t["groups"][0], d["lam"], err)
            assert dg[i]["dt"] == pytest.approx(rdiag[i]["dt"], rel=1e-5)
            assert dg[i]["E"] == pytest.approx(rdiag[i]["E"], rel=1e-5)
            assert dg[i]["P"] == pytest.approx(math.exp(d["lam"]) * d["eps_bar"], rel=1e-6)
        ens.close()
    parity_log("128^3 one RK3 step, worst rel L2 over %d variants x 3 members" % len(variants), worst, 1e-5)


# ---------------------------------------------------------------------------
# N = 256, 384, 512: stored oracle samples
# ---------------------------------------------------------------------------
def load_golden(N):
    path = os.path.join(GOLDEN, "one_step_%d.npz" % N)
    if not os.path.exists(path):
        pytest.fail("missing %s: run tests/golden/make_oracle_goldens.py one_step %d" % (path, N))
    z = np.load(path)
    cases = []
    for ci in range(int(z["cases"])):
        cases.append(dict(desc=json.loads(str(z["c%d_desc" % ci])), modes=z["c%d_modes" % ci],
                          values=z["c%d_values" % ci], diag=z["c%d_diag" % ci], counts=z["c%d_counts" % ci],
                          moments=z["c%d_moments" % ci]))
    return cases


@pytest.mark.parametrize("N", [256, 384, 512])
def test_one_step_large_every_variant_matches_stored_oracle(E, N, parity_log):
    cases = load_golden(N)
    worst = 0.0
    for case in cases:
        d = case["desc"]
        m = lib_member(E, d)
        modes = case["modes"]
        ix, iy, iz = modes[:, 0], modes[:, 1], modes[:, 2]
        probe = E.Ensemble([m], hist=E.hist_spec(nu_norm=d["nu"], **HIST))
        variants = tunings(E, probe, N)
        probe.close()
        for vi, t in enumerate(variants):
            ens = E.Ensemble([m], hist=E.hist_spec(nu_norm=d["nu"], **HIST))
            ens.set_tuning(t)
            ens.step(1)
            f = ens.field(0)
            got = f[:, ix, iy, iz]
            del f
            err = rel(got, case["values"])
            worst = max(worst, err)
            assert err < 1e-5, (d["name"], t["groups"][0], err)
            g = ens.diagnostics()[0]
            t_, dt, E_, diss, EB, P, umax = case["diag"]
            assert g["dt"] == pytest.approx(dt, rel=1e-5)
            assert g["E"] == pytest.approx(E_, rel=1e-5)
            assert g["P"] == pytest.approx(math.exp(d["lam"]) * d["eps_bar"], rel=1e-6)
            if vi == 0:
                parity_log("%d^3 %s dt rel error" % (N, d["name"]), abs(g["dt"] / dt - 1), 1e-5)
                parity_log("%d^3 %s E rel error" % (N, d["name"]), abs(g["E"] / E_ - 1), 1e-5)
                parity_log("%d^3 %s dissipation rel error" % (N, d["name"]), abs(g["diss"] / diss - 1), None)
                ens.gradient_stats(accumulate=False)
                counts, mom = ens.stats()
                check_stats(counts[0], case["counts"], N ** 3, parity_log, "%d^3 %s statistics" % (N, d["name"]))
                for k in list(range(0, 36, 4)) + [38, 39]:
                    assert mom[0, k] == pytest.approx(case["moments"][k], rel=1e-4), k
                mrel = max(abs(mom[0, k] / case["moments"][k] - 1) for k in list(range(0, 36, 4)) + [38, 39])
                parity_log("%d^3 %s second moments / eps / omega^2 sums, max rel error" % (N, d["name"]), mrel, 1e-4)
            ens.close()
    parity_log("%d^3 one RK3 step, worst sampled rel L2 over variants and members" % N, worst, 1e-5)
