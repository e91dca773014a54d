"""Failure detection on the GPU without a fault: a bounded device wait that
runs out.

ens_test_skip_copy arms one ens_step_nograph call so that the persistent z
pass issues no bulk copy for one row group of one member and waits for that
group's barrier only a few hundred polls: the wait gives up with nothing in
flight (every copy that was issued is still waited for with the full limit),
the member is flagged and ens_diagnostics returns ENS_ETIMEOUT.  Nothing
hangs and the context stays usable; a fresh context afterwards steps as
usual.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ENS_ETIMEOUT = 5


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


def members(E, N):
    return [E.Member(N=N, nu=0.02, lam=l, k_lo=1, k_hi=2, dt=0.005, rk_order=3, seed=90 + i)
            for i, l in enumerate((-0.5, 0.0, 0.6))]


def oracle_step(m, nsteps):
    om = O.Member(N=m.N, nu=m.nu, lam=m.lam, eps_bar=m.eps_bar, k_lo=m.k_lo, k_hi=m.k_hi, dt=m.dt, cfl=m.cfl,
                  dt_max=m.dt_max, rk_order=m.rk_order, seed=m.seed, init_energy=m.init_energy)
    uh = O.initial_field(om)
    assert O.step(om, uh, nsteps)[0] == 0
    return uh


@pytest.mark.parametrize("N", [32, 64])
def test_bounded_wait_runs_out_and_is_reported(E, N):
    ms = members(E, N)
    ens = E.Ensemble(ms)
    assert ens.tuning()["groups"][0]["z_variant"] == 0     # the persistent TMA z pass
    E.ens_test_skip_copy(ens.ctx, 2, 256)
    ens.step(1, graph=False)
    diags, status = E.ens_diagnostics(ens.ctx, len(ms), raise_on_flag=False)
    assert status == ENS_ETIMEOUT
    assert diags[2]["flags"] & 4
    assert not (diags[0]["flags"] & 4) and not (diags[1]["flags"] & 4)
    # the members before the flagged one went through untouched
    for i in (0, 1):
        assert rel(ens.field(i), oracle_step(ms[i], 1)) < 1e-5, i
    # the hook is one-shot, and its argument errors are not sticky
    with pytest.raises(E.EnsError) as err:
        E.ens_test_skip_copy(ens.ctx, 3, 256)
    assert err.value.status == 1
    with pytest.raises(E.EnsError):
        E.ens_test_skip_copy(ens.ctx, 0, 0)
    ens.step(1, graph=False)
    diags2, status2 = E.ens_diagnostics(ens.ctx, len(ms), raise_on_flag=False)
    assert diags2[0]["steps"] == 2 and not (diags2[0]["flags"] & 4)
    ens.close()
    # a fresh context steps normally and matches the oracle
    fresh = E.Ensemble(ms)
    fresh.step(2)
    diags3, status3 = E.ens_diagnostics(fresh.ctx, len(ms), raise_on_flag=False)
    assert status3 == 0 and all(d["flags"] == 0 for d in diags3)
    for i, m in enumerate(ms):
        assert rel(fresh.field(i), oracle_step(m, 2)) < 1e-5, i
    fresh.close()


def test_skip_hook_refuses_the_row_group_z_pass(E):
    ens = E.Ensemble(members(E, 32))
    t = ens.tuning()
    t["groups"][0]["z_variant"] = 1
    ens.set_tuning(t)
    with pytest.raises(E.EnsError) as err:
        E.ens_test_skip_copy(ens.ctx, 0, 256)
    assert err.value.status == 1
    ens.step(1)
    assert E.ens_diagnostics(ens.ctx, 3, raise_on_flag=False)[1] == 0
    ens.close()
