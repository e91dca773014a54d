"""The persistent stage kernel: every member of every grid size (128, 256,
384) advancing one RK stage in one launch, against the graph of per-pass
launches and the FP64 oracle.

Members of the uneven-size batch (nu per member for k_max eta >= 1.5, band
[6, 8], IF-RK3, CFL 0.2).  The persistent kernel runs the same pass bodies as
the separate kernels with 16-column tiles, 16 threads per FFT line, the
default z warp plan and the fused last pass, with those variants installed
in the graph path the fields agree to FP32 rounding: the z pass pairs the
n_z rows of a warp's stream into one complex line, and the persistent
kernel's warps stream over other rows (so the rounding of a row's transform
depends on another partner row), and the 128^3 members run their y passes
on the second FFT plan.  Every member matches the oracle after one step
(relative L2 <= 1e-5); the captured graph and direct launches of the
persistent kernel agree bit for bit.
"""
import json
import math

import numpy as np
import pytest

import ens_inputs as I
import oracle as O

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def picks():
    ds = I.uneven_batch()
    by = {}
    for d in ds:
        by.setdefault(d["N"], []).append(d)
    return [by[128][0], by[128][-1], by[256][0], by[384][0]]


def lib_member(E, d):
    return E.Member(N=d["N"], nu=d["nu"], lam=d["lam"], eps_bar=d["eps_bar"], k_lo=d["k_lo"], k_hi=d["k_hi"],
                    dt=d["dt"], cfl=d["cfl"], dt_max=d["dt_max"], rk_order=d["rk_order"], seed=d["seed"],
                    init_energy=d["init_energy"])


def oracle_member(d):
    return O.Member(N=d["N"], nu=d["nu"], lam=d["lam"], eps_bar=d["eps_bar"], k_lo=d["k_lo"], k_hi=d["k_hi"],
                    dt=d["dt"], cfl=d["cfl"], dt_max=d["dt_max"], rk_order=d["rk_order"], seed=d["seed"],
                    init_energy=d["init_energy"])


def graph_tuning_like_persistent(t):
    t = json.loads(json.dumps(t))
    t["persistent"] = 0
    for g in t["groups"]:
        g.update(tile_x=16, tile_y=16, plan_x=1 if g["N"] == 128 else 0, fx_split=0, z_variant=0)
    return t


def test_persistent_matches_graph_and_oracle(E, parity_log):
    ds = picks()
    ms = [lib_member(E, d) for d in ds]
    a, b = E.Ensemble(ms), E.Ensemble(ms)
    ta = graph_tuning_like_persistent(a.tuning())
    a.set_tuning(ta)
    tb = b.tuning()
    tb["persistent"] = 1
    b.set_tuning(tb)
    assert b.tuning()["persistent"] == 1
    assert E.ens_kernels_per_step(b.ctx) == 3
    a.step(1)
    b.step(1)            # the captured graph of three cooperative launches
    da, db = a.diagnostics(), b.diagnostics()
    worst = 0.0
    for i, d in enumerate(ds):
        fa, fb = a.field(i), b.field(i)
        assert rel(fb, fa) < 1e-6, i
        assert db[i]["dt"] == pytest.approx(da[i]["dt"], rel=1e-6)
        assert db[i]["E"] == pytest.approx(da[i]["E"], rel=1e-6)
        om = oracle_member(d)
        if d["N"] <= 256:
            uh = O.initial_field(om)
            assert O.step(om, uh, 1)[0] == 0
            err = rel(fb, uh)
            worst = max(worst, err)
            assert err < 1e-5, (i, d["N"], err)
        assert db[i]["P"] == pytest.approx(math.exp(d["lam"]) * d["eps_bar"], rel=1e-6)
        assert db[i]["steps"] == 1 and db[i]["flags"] == 0
    parity_log("persistent stage kernel, one RK3 step (128^3, 256^3), worst rel L2 vs the oracle", worst, 1e-5)
    # direct launches give the same as the graph, over two more steps
    c = E.Ensemble(ms)
    c.set_tuning(tb)
    c.step(1)
    b.step(2)
    c.step(2, graph=False)
    for i in range(len(ds)):
        assert np.array_equal(b.field(i), c.field(i)), i
    for e in (a, b, c):
        e.close()


def test_persistent_384_member_matches_stored_oracle(E, parity_log):
    """The 384^3 member against the stored oracle step of the same member
    (tests/golden/one_step_384.npz, case 0)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "one_step_384.npz")
    if not os.path.exists(path):
        pytest.fail("missing %s: run tests/golden/make_oracle_goldens.py one_step 384" % path)
    z = np.load(path)
    d = json.loads(str(z["c0_desc"]))
    assert d["N"] == 384 and d["seed"] == picks()[3]["seed"]
    m = lib_member(E, d)
    e = E.Ensemble([m, lib_member(E, picks()[0])])
    t = e.tuning()
    t["persistent"] = 1
    e.set_tuning(t)
    e.step(1)
    modes = z["c0_modes"]
    got = e.field(0)[:, modes[:, 0], modes[:, 1], modes[:, 2]]
    err = parity_log("persistent stage kernel, 384^3 one RK3 step, sampled rel L2 vs the stored oracle",
                     rel(got, z["c0_values"]), 1e-5)
    assert err < 1e-5
    assert e.diagnostics()[0]["dt"] == pytest.approx(float(z["c0_diag"][1]), rel=1e-5)
    e.close()


def test_persistent_refused_for_other_sizes(E):
    e = E.Ensemble([E.Member(N=64, nu=0.02, k_lo=1, k_hi=2), E.Member(N=128, nu=0.02, k_lo=1, k_hi=2)])
    t = e.tuning()
    t["persistent"] = 1
    with pytest.raises(E.EnsError) as err:
        e.set_tuning(t)
    assert err.value.status == 1
    assert e.tuning()["persistent"] == 0
    e.step(1)
    e.close()
