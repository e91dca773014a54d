"""Autotuner and pass variants through the C ABI.

Every tuning variant (column tiles 8/16 of the x and y passes, persistent or
row-group z pass, parallel or chained grid-size groups) advances the members
to the oracle's state within the one-step tolerance (relative L2 <= 1e-5),
and agrees with the default variant to FP32 rounding of the energy sums.
ens_autotune leaves the member state untouched, installs a valid tuning, and
the cached tuning round-trips through ens_set_tuning.
"""
import json

import numpy as np
import pytest

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


def members(E):
    return [E.Member(N=n, nu=0.03, lam=0.3 * i - 0.6, k_lo=1, k_hi=2, dt=-1, cfl=0.2, dt_max=0.01, rk_order=3,
                     seed=60 + i) for i, n in enumerate([32, 64, 32, 16])]


def oracle_member(m):
    return O.Member(N=m.N, nu=m.nu, lam=m.lam, eps_bar=m.eps_bar, k_lo=m.k_lo, k_hi=m.k_hi, dt=m.dt, cfl=m.cfl,
                    dt_max=m.dt_max, rk_order=m.rk_order, seed=m.seed, init_energy=m.init_energy)


def variants(base):
    out = []
    for tx in (16, 8):
        for ty in (16, 8):
            for zv in (0, 1):
                t = json.loads(json.dumps(base))
                for g in t["groups"]:
                    g.update(tile_x=tx, tile_y=ty, z_variant=zv)
                out.append(t)
    t = json.loads(json.dumps(base))
    t["parallel_groups"] = 0
    out.append(t)
    t = json.loads(json.dumps(base))
    for g in t["groups"]:
        g["z_ctas_per_sm"] = 1
    out.append(t)
    for tx in (16, 8):
        t = json.loads(json.dumps(base))
        for g in t["groups"]:
            g.update(fx_split=1, tile_x=tx)
        out.append(t)
    return out


def test_default_tuning(E):
    ens = E.Ensemble(members(E))
    t = ens.tuning()
    assert [g["N"] for g in t["groups"]] == [16, 32, 64]
    assert t["parallel_groups"] == 1
    for g in t["groups"]:
        assert g["tile_x"] == 16 and g["tile_y"] == 16 and g["z_variant"] == 0 and g["z_ctas_per_sm"] >= 1
    ens.close()


def test_every_variant_matches_oracle(E):
    ms = members(E)
    refs = []
    for m in ms:
        om = oracle_member(m)
        uh = O.initial_field(om)
        O.step(om, uh, 1)
        refs.append(uh)
    base = E.Ensemble(ms)
    base.step(1)
    base_fields = [base.field(i) for i in range(len(ms))]
    for t in variants(base.tuning()):
        ens = E.Ensemble(ms)
        ens.set_tuning(t)
        assert ens.tuning()["groups"] == t["groups"]
        ens.step(1)
        for i in range(len(ms)):
            f = ens.field(i)
            assert rel(f, refs[i]) < 1e-5, (t, i)
            assert rel(f, base_fields[i]) < 1e-6, (t, i)
        ens.close()
    base.close()


def test_x_plan_variant_matches_oracle(E):
    """The second FFT plan of the x passes (N = 128: 8x2x8 on 16 threads per
    line) with both column tiles, against the oracle after one RK3 step."""
    m = E.Member(N=128, nu=0.01, lam=0.7, k_lo=1, k_hi=2, dt=-1, cfl=0.2, dt_max=0.01, rk_order=3, seed=71)
    om = oracle_member(m)
    ref = O.initial_field(om)
    O.step(om, ref, 1)
    base = E.Ensemble([m])
    base.step(1)
    f0 = base.field(0)
    base.close()
    for plan in (1,):
        for tx in (16, 8):
            ens = E.Ensemble([m])
            t = ens.tuning()
            t["groups"][0].update(plan_x=plan, tile_x=tx)
            ens.set_tuning(t)
            ens.step(1)
            f = ens.field(0)
            assert rel(f, ref) < 1e-5, (plan, tx)
            assert rel(f, f0) < 1e-6, (plan, tx)
            ens.close()
    # sizes without a second plan refuse plan_x = 1
    ens = E.Ensemble(members(E))
    t = ens.tuning()
    t["groups"][0]["plan_x"] = 1
    with pytest.raises(E.EnsError):
        ens.set_tuning(t)
    ens.close()


def test_z_plan_variant_matches_oracle(E):
    """The persistent z pass with the two-pass 16 x 16 warp plan (N = 256,
    z_variant 2) against the oracle after one RK3 step, and against the
    default plan."""
    m = E.Member(N=256, nu=0.005, lam=0.4, k_lo=6, k_hi=8, dt=-1, cfl=0.2, rk_order=3, seed=2027)
    om = oracle_member(m)
    ref = O.initial_field(om)
    O.step(om, ref, 1)
    base = E.Ensemble([m])
    base.step(1)
    f0 = base.field(0)
    base.close()
    ens = E.Ensemble([m])
    t = ens.tuning()
    t["groups"][0].update(z_variant=2, z_ctas_per_sm=1)
    ens.set_tuning(t)
    ens.step(1)
    f = ens.field(0)
    assert rel(f, ref) < 1e-5
    assert rel(f, f0) < 1e-6
    ens.close()
    # other sizes refuse it
    ens = E.Ensemble(members(E))
    t = ens.tuning()
    t["groups"][1]["z_variant"] = 2
    with pytest.raises(E.EnsError):
        ens.set_tuning(t)
    ens.close()


def test_invalid_tuning_rejected_and_context_usable(E):
    ens = E.Ensemble(members(E))
    good = ens.tuning()
    for bad in ({"tile_x": 4}, {"tile_y": 32}, {"z_variant": 3}, {"z_ctas_per_sm": 0}, {"z_ctas_per_sm": 99},
                {"N": 128}):
        t = json.loads(json.dumps(good))
        t["groups"][1].update(bad)
        with pytest.raises(E.EnsError):
            ens.set_tuning(t)
    t = json.loads(json.dumps(good))
    t["groups"] = t["groups"][:2]
    with pytest.raises(E.EnsError):
        ens.set_tuning(t)
    assert ens.tuning()["groups"] == good["groups"]
    ens.step(1)
    ens.diagnostics()
    ens.close()


@pytest.mark.parametrize("change", [{"tile_x": 8}, {"fx_split": 1}])
def test_update_variants_keep_energy_sums_over_several_steps(E, change):
    """tile_x = 8 doubles the update pass's CTA partials of the FP64 energy
    sums and fx_split = 1 moves them to the split update launch; after three
    steps the forcing amplitude (from E_B) still gives the exact injected
    power and the fields follow the oracle."""
    ms = members(E)
    ens = E.Ensemble(ms)
    t = ens.tuning()
    for g in t["groups"]:
        g.update(change)
    ens.set_tuning(t)
    ens.step(3)
    for i, (m, d) in enumerate(zip(ms, ens.diagnostics())):
        assert d["P"] == pytest.approx(np.exp(m.lam) * m.eps_bar, rel=1e-5)
        om = oracle_member(m)
        uh = O.initial_field(om)
        O.step(om, uh, 3)
        assert rel(ens.field(i), uh) < 1e-4
    ens.close()


def test_autotune_preserves_state_and_caches(E, tmp_path):
    ms = members(E)
    ens = E.Ensemble(ms)
    ens.step(2)
    before = [ens.field(i) for i in range(len(ms))]
    d0 = ens.diagnostics()
    t = ens.autotune(steps=2, cache=str(tmp_path / "tune.json"))
    assert not t["cached"] and t["trials"] >= 4 and t["ms_per_step"] > 0
    for i in range(len(ms)):
        assert np.array_equal(ens.field(i), before[i])
    d1 = ens.diagnostics()
    assert [d["t"] for d in d1] == [d["t"] for d in d0]
    assert [d["steps"] for d in d1] == [d["steps"] for d in d0]
    installed = ens.tuning()
    assert installed["groups"] == t["groups"] and installed["parallel_groups"] == t["parallel_groups"]
    # the tuned context keeps stepping like its oracle members
    ens.step(1)
    for i, m in enumerate(ms):
        om = oracle_member(m)
        uh = O.initial_field(om)
        O.step(om, uh, 3)
        assert rel(ens.field(i), uh) < 1e-4
    # a second context of the same members installs the cached tuning
    other = E.Ensemble(ms)
    t2 = other.autotune(cache=str(tmp_path / "tune.json"))
    assert t2["cached"] and other.tuning()["groups"] == t["groups"]
    other.close()
    ens.close()


def test_warp_group_last_pass_equals_fused(E):
    """The last pass in two overlapping warp groups (fx_split 2, N = 256)
    gives, bit for bit, the fields and energy sums of the fused pass on
    16-column tiles, over two steps with CFL time steps; and ens_step_host
    (members in chunks of one) runs it too.  Chunked launches agree with the
    whole group's launch to FP32 rounding, not bit for bit: the z pass
    pairs the n_z rows of a warp's stream of rows, and the stream depends on
    the members in the launch."""
    ms = [E.Member(N=256, nu=0.005, lam=l, k_lo=6, k_hi=8, dt=-1, cfl=0.2, rk_order=3, seed=300 + i)
          for i, l in enumerate((-1.0, 0.4, 2.1))]
    a, b = E.Ensemble(ms), E.Ensemble(ms)
    ta = a.tuning()
    ta["groups"][0].update(fx_split=0, tile_x=16, plan_x=0)
    a.set_tuning(ta)
    tb = b.tuning()
    tb["groups"][0].update(fx_split=2, tile_x=16, plan_x=0)
    b.set_tuning(tb)
    assert b.tuning()["groups"][0]["fx_split"] == 2
    a.step(2)
    b.step(2)
    da, db = a.diagnostics(), b.diagnostics()
    for i in range(len(ms)):
        assert np.array_equal(a.field(i), b.field(i)), i
        for k in ("dt", "E", "diss", "EB", "P"):
            assert da[i][k] == db[i][k], (i, k)
    nbytes = E.ens_state_bytes(b.ctx)
    host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    E.ens_get_state(b.ctx, host.data_ptr(), nbytes)
    ref = host.clone()
    E.ens_step_host(b.ctx, host.data_ptr(), host.data_ptr(), nbytes, 1)
    E.ens_set_state(a.ctx, ref.data_ptr(), nbytes)
    a.step(1)
    E.ens_set_state(b.ctx, host.data_ptr(), nbytes)
    for i in range(len(ms)):
        fa, fb = a.field(i), b.field(i)
        assert np.linalg.norm(fb - fa) <= 1e-6 * np.linalg.norm(fa), i
    a.close()
    b.close()
