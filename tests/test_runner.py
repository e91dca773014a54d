"""Run-driver policy on the host (no GPU): transient cut, snapshot cadence,
checkpoints, JSON-lines log, and rollback of a member that goes non-finite
with a smaller CFL number.  The ensemble is a fake with the library's
method names; the failure is made on the host (a flag the fake raises)."""
import copy
import json
from types import SimpleNamespace

import pytest

from paper_2506_23712_gb300 import runner


class FakeEnsemble:
    """Members blow up (non-finite flag) whenever their CFL number is above
    `unstable_above` once `blowup_step` steps have been taken."""

    def __init__(self, cfls, unstable_above=None, blowup_step=0):
        self.members = [SimpleNamespace(dt=-1.0, cfl=c, dt_max=0.0) for c in cfls]
        self.cfl = list(cfls)
        self.t = 0
        self.unstable_above = unstable_above
        self.blowup_step = blowup_step
        self.stats_calls = []
        self.saved = None
        self.calls = []

    def step(self, n):
        self.t += n
        self.calls.append(("step", n))

    def diagnostics(self, raise_on_flag=True):
        out = []
        for c in self.cfl:
            bad = self.unstable_above is not None and c > self.unstable_above and self.t >= self.blowup_step
            out.append({"t": float(self.t), "flags": 1 if bad else 0})
        return out

    def gradient_stats(self, accumulate=True):
        self.stats_calls.append((self.t, accumulate))

    def save(self, path):
        self.saved = (self.t, list(self.stats_calls), list(self.cfl))
        self.calls.append(("save", self.t))

    def load(self, path):
        self.t, stats, cfl = copy.deepcopy(self.saved)
        self.stats_calls = stats
        self.cfl = cfl
        self.calls.append(("load", self.t))

    def set_timestep(self, i, dt, cfl, dt_max):
        self.cfl[i] = cfl
        self.calls.append(("set", i, cfl))


def test_cadence_transient_and_log(tmp_path):
    ens = FakeEnsemble([0.2, 0.2])
    log = tmp_path / "run.jsonl"
    rep = runner.run(ens, 50, transient=20, stats_every=10, log_path=str(log))
    assert rep.steps_done == 50 and rep.snapshots == 3
    # first snapshot resets the statistics, later ones accumulate
    assert ens.stats_calls == [(30, False), (40, True), (50, True)]
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    assert [l["step"] for l in lines] == [10, 20, 30, 40, 50]


def test_nonfinite_member_rolls_back_with_smaller_cfl(tmp_path):
    ens = FakeEnsemble([0.2, 0.4, 0.2], unstable_above=0.25, blowup_step=25)
    ck = str(tmp_path / "ens.ckpt")
    log = tmp_path / "run.jsonl"
    rep = runner.run(ens, 60, transient=0, stats_every=10, checkpoint_every=20, checkpoint_path=ck,
                     log_path=str(log))
    assert rep.failed == [] and rep.steps_done == 60
    assert rep.rollbacks == 1 and rep.retried == {1: 1}
    assert ens.cfl == [0.2, 0.2, 0.2]
    # rolled back to the checkpoint at step 20, then continued
    assert ("load", 20) in ens.calls and ("set", 1, 0.2) in ens.calls
    # snapshots at 10, 20 before the failure; 30..60 after; none lost or doubled
    assert [t for t, _ in ens.stats_calls] == [10, 20, 30, 40, 50, 60]
    events = [json.loads(x) for x in log.read_text().splitlines() if "event" in x]
    assert events and events[0]["to_step"] == 20 and events[0]["members"] == [1]


def test_member_that_stays_unstable_is_reported(tmp_path):
    ens = FakeEnsemble([0.2, 0.9], unstable_above=0.1, blowup_step=5)
    rep = runner.run(ens, 40, stats_every=10, checkpoint_path=str(tmp_path / "c"), max_retries=2)
    # member 0 recovers at CFL 0.1; member 1 (0.9 -> 0.45 -> 0.225) does not
    assert rep.failed == [1] and rep.steps_done == 0
    assert rep.retried == {0: 1, 1: 2} and ens.cfl == pytest.approx([0.1, 0.225])


def test_without_checkpoint_a_failure_stops_the_run():
    ens = FakeEnsemble([0.2, 0.4], unstable_above=0.25, blowup_step=15)
    rep = runner.run(ens, 40, stats_every=10)
    assert rep.failed == [1] and rep.steps_done == 10 and rep.rollbacks == 0


def test_bad_arguments():
    with pytest.raises(ValueError):
        runner.run(FakeEnsemble([0.2]), 10, stats_every=0)
