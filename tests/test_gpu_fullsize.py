"""Full-size parity in the benchmark's launch configuration: the 64-member
256^3 ensemble (nu = 0.005, band [6, 8], lambda ~ N(0, 2^2) clipped,
IF-RK3, CFL 0.2) advanced one step by the captured graph with the
autotuner's choice installed, exactly as bench.py runs it; sampled members
(the extreme and the central lambda) against the FP64 oracle run on their
own: relative L2 <= 1e-5 after one step, the same CFL step, and the
gradient statistics of each of them within 2% in every bin above 1000 counts.
Ten steps of the same launch configuration against the oracle's ten steps of
the central member (stored, ``tests/golden/ten_steps_256.npz``, sampled
modes): relative L2 <= 1e-4 (the one-step bound grows with the steps; the
32^3 runs are held to 1e-3 after 100), the CFL step and energy of every step
within 1e-5.
"""
import json
import os

import numpy as np
import pytest

import ens_inputs as I
import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

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


def test_benchmark_ensemble_sampled_members_match_oracle(E, parity_log):
    ds = I.ensemble_256()
    ms = [E.Member(N=d["N"], nu=d["nu"], lam=d["lam"], eps_bar=d["eps_bar"], k_lo=d["k_lo"], k_hi=d["k_hi"],
                   dt=d["dt"], cfl=d["cfl"], dt_max=d["dt_max"], rk_order=d["rk_order"], seed=d["seed"],
                   init_energy=d["init_energy"]) for d in ds]
    kw = dict(qr_bins=64, q_lim=10.0, r_lim=10.0, tail_bins=256, tail_lo=-8.0, tail_hi=8.0, eps_norm=0.1,
              nu_norm=0.005)
    ens = E.Ensemble(ms, hist=E.hist_spec(**kw))
    ens.autotune(steps=1)
    ens.step(1)
    diags = ens.diagnostics()
    lams = np.array([d["lam"] for d in ds])
    picks = sorted({int(np.argmin(lams)), int(np.argmax(lams)), int(np.argmin(np.abs(lams)))})
    for i in picks:
        d = ds[i]
        om = O.Member(N=d["N"], nu=d["nu"], lam=d["lam"], eps_bar=d["eps_bar"], k_lo=d["k_lo"], k_hi=d["k_hi"],
                      dt=d["dt"], cfl=d["cfl"], dt_max=d["dt_max"], rk_order=d["rk_order"], seed=d["seed"],
                      init_energy=d["init_energy"])
        uh = O.initial_field(om)
        st, od = O.step(om, uh, 1)
        assert st == 0
        err = parity_log("256^3 benchmark ensemble (autotuned), member lambda=%.3f: field after 1 step, rel L2"
                         % d["lam"], rel(ens.field(i), uh), 1e-5)
        assert err < 1e-5, (i, d["lam"])
        parity_log("256^3 benchmark member lambda=%.3f: dt rel error" % d["lam"], abs(diags[i]["dt"] / od["dt"] - 1),
                   1e-5)
        parity_log("256^3 benchmark member lambda=%.3f: E rel error" % d["lam"], abs(diags[i]["E"] / od["E"] - 1),
                   None)
        assert diags[i]["dt"] == pytest.approx(od["dt"], rel=1e-5)
        # gradient statistics of the smallest, central and largest lambda
        if i == picks[0]:
            ens.gradient_stats(accumulate=False)
            counts, _ = ens.stats()
        rc, _ = O.gradient_stats(uh, d["nu"], O.HistSpec(**kw))
        c, r = counts[i].astype(np.int64), rc.astype(np.int64)
        assert c[-2] == r[-2] == d["N"] ** 3
        big = r > 1000
        assert big.sum() >= 50
        dev = float((np.abs(c[big] - r[big]) / r[big]).max())
        parity_log("256^3 benchmark member lambda=%.3f: statistics max bin deviation (bins > 1000)" % d["lam"],
                   dev, 0.02)
        assert dev <= 0.02
    ens.close()


def test_benchmark_ensemble_ten_steps_match_stored_oracle(E, parity_log):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ten_steps_256.npz")
    if not os.path.exists(path):
        pytest.fail("missing %s: run tests/golden/make_oracle_goldens.py ten_steps" % path)
    z = np.load(path)
    gd = json.loads(str(z["desc"]))
    ds = I.ensemble_256()
    i = gd["index"]
    assert ds[i]["seed"] == gd["seed"] and ds[i]["lam"] == gd["lam"]
    ms = [E.Member(N=d["N"], nu=d["nu"], lam=d["lam"], eps_bar=d["eps_bar"], k_lo=d["k_lo"], k_hi=d["k_hi"],
                   dt=d["dt"], cfl=d["cfl"], dt_max=d["dt_max"], rk_order=d["rk_order"], seed=d["seed"],
                   init_energy=d["init_energy"]) for d in ds]
    ens = E.Ensemble(ms, hist=E.hist_spec(nu_norm=0.005))
    ens.autotune(steps=1)
    worst_dt = worst_E = 0.0
    for s in range(10):
        ens.step(1)
        g = ens.diagnostics()[i]
        t_, dt, E_, diss, EB, P, umax = z["diags"][s]
        worst_dt = max(worst_dt, abs(g["dt"] / dt - 1))
        worst_E = max(worst_E, abs(g["E"] / E_ - 1))
    modes = z["modes"]
    got = ens.field(i)[:, modes[:, 0], modes[:, 1], modes[:, 2]]
    err = parity_log("256^3 benchmark ensemble (autotuned), central member: field after 10 steps, sampled rel L2",
                     rel(got, z["values"]), 1e-4)
    parity_log("256^3 benchmark ensemble, central member: dt over 10 steps, max rel error", worst_dt, 1e-5)
    parity_log("256^3 benchmark ensemble, central member: E over 10 steps, max rel error", worst_E, 1e-5)
    assert err < 1e-4
    assert worst_dt < 1e-5 and worst_E < 1e-5
    ens.close()
