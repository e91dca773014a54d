"""Checkpoint / resume through the C ABI: an ensemble saved after some steps
and loaded into a fresh context with the same members continues bit for bit
like the saved one (fields, run state, statistics); foreign, truncated or
corrupted files are refused without touching the context."""
import os

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


def members(E, lam0=-0.4):
    return [E.Member(N=n, nu=0.03, lam=lam0 + 0.4 * i, k_lo=1, k_hi=2, dt=-1, cfl=0.2, dt_max=0.01, rk_order=3,
                     seed=90 + i) for i, n in enumerate([32, 16, 32])]


def hist(E):
    return E.hist_spec(qr_bins=8, tail_bins=16, nu_norm=0.03, grad_bins=12, grad_lim=6.0)


def test_resume_is_bit_identical(E, tmp_path):
    ms = members(E)
    a = E.Ensemble(ms, hist=hist(E))
    a.step(3)
    a.gradient_stats(accumulate=False)
    path = str(tmp_path / "ens.ckpt")
    a.save(path)
    assert os.path.exists(path) and not os.path.exists(path + ".tmp")
    a.step(2)
    a.gradient_stats(accumulate=True)
    b = E.Ensemble(ms, hist=hist(E))
    b.load(path)
    b.step(2)
    b.gradient_stats(accumulate=True)
    for i in range(len(ms)):
        assert np.array_equal(a.field(i), b.field(i)), i
    da, db = a.diagnostics(), b.diagnostics()
    for x, y in zip(da, db):
        assert x == y
    ca, ma = a.stats()
    cb, mb = b.stats()
    assert np.array_equal(ca, cb) and np.array_equal(ma, mb)
    # a tuned context resumes the same checkpoint (tile_x = 8 doubles the
    # energy partials; the loaded run state follows the installed tuning)
    c = E.Ensemble(ms, hist=hist(E))
    t = c.tuning()
    for g in t["groups"]:
        g["tile_x"] = 8
    c.set_tuning(t)
    c.load(path)
    c.step(2)
    for i, m in enumerate(ms):
        d = c.diagnostics()[i]
        assert d["P"] == pytest.approx(np.exp(m.lam) * m.eps_bar, rel=1e-5)
        f, g = c.field(i), a.field(i)
        assert np.linalg.norm(f - g) <= 1e-6 * np.linalg.norm(g)
    for e in (a, b, c):
        e.close()


def test_load_refuses_bad_files(E, tmp_path):
    ms = members(E)
    a = E.Ensemble(ms, hist=hist(E))
    a.step(1)
    path = str(tmp_path / "ens.ckpt")
    a.save(path)
    before = [a.field(i) for i in range(len(ms))]
    with pytest.raises(E.EnsError):
        a.load(str(tmp_path / "missing.ckpt"))
    # other members (lambda differs)
    other = E.Ensemble(members(E, lam0=0.1), hist=hist(E))
    with pytest.raises(E.EnsError):
        other.load(path)
    other.close()
    # truncated
    raw = open(path, "rb").read()
    bad = str(tmp_path / "bad.ckpt")
    with open(bad, "wb") as f:
        f.write(raw[: len(raw) // 2])
    with pytest.raises(E.EnsError):
        a.load(bad)
    # one flipped byte in the payload
    flipped = bytearray(raw)
    flipped[len(raw) - 100] ^= 0x40
    with open(bad, "wb") as f:
        f.write(bytes(flipped))
    with pytest.raises(E.EnsError):
        a.load(bad)
    # the context is untouched and still steps
    for i in range(len(ms)):
        assert np.array_equal(a.field(i), before[i])
    a.step(1)
    a.diagnostics()
    a.close()


def test_run_driver_recovers_a_nonfinite_member(E, tmp_path):
    """The run driver on the library: a member made non-finite on the host
    side (NaN written into its spectrum once, as a stand-in for a blow-up)
    rolls the ensemble back to the last checkpoint with that member's CFL
    number halved (ens_set_timestep) and the run completes; the other members
    end exactly where an undisturbed run ends."""
    from paper_2506_23712_gb300 import runner
    ms = members(E)

    class Injecting:
        def __init__(self, ens):
            self.ens, self.members, self.done = ens, ens.members, False

        def step(self, n):
            self.ens.step(n)
            if not self.done and self.ens.diagnostics()[0]["steps"] >= 6:
                f = self.ens.field(1)
                f[0, 1, 1, 1] = np.nan
                self.ens.set_field(1, f)
                self.ens.step(1)          # the NaN spreads through the step
                self.done = True

        def __getattr__(self, k):
            return getattr(self.ens, k)

    a = E.Ensemble(ms, hist=hist(E))
    rep = runner.run(Injecting(a), 12, stats_every=3, checkpoint_every=3,
                     checkpoint_path=str(tmp_path / "run.ckpt"), log_path=str(tmp_path / "run.jsonl"))
    assert rep.failed == [] and rep.rollbacks == 1 and rep.retried == {1: 1} and rep.steps_done == 12
    d = a.diagnostics()
    assert all(x["flags"] == 0 for x in d)
    b = E.Ensemble(ms, hist=hist(E))
    b.step(12)
    for i in (0, 2):
        assert np.array_equal(a.field(i), b.field(i)), i
    a.close()
    b.close()
