"""Run driver for an ensemble: transient cut, statistics cadence, periodic
checkpoints, a JSON-lines diagnostics log, and recovery from members that
go non-finite.

The paper discards an initial transient of every member run and then
accumulates statistics over the rest (Sec. IV); the driver does the same with
`transient` steps and a snapshot every `stats_every` steps.  A member that
goes non-finite (the library's per-member flag, ENS_ENONFINITE) rolls the
whole ensemble back to the last checkpoint, that member's CFL number (or
fixed dt) is scaled by `retry_factor`, and the run continues; after
`max_retries` failed attempts of one member the driver stops and reports it.
Host policy only: every step, snapshot and reload is a library call.
"""
from __future__ import annotations

import json
import time
from dataclasses import dataclass, field
from typing import List, Optional

FLAG_NONFINITE = 1


@dataclass
class RunReport:
    steps_done: int = 0
    snapshots: int = 0
    checkpoints: int = 0
    rollbacks: int = 0
    retried: dict = field(default_factory=dict)      # member -> attempts
    failed: List[int] = field(default_factory=list)  # members that exhausted their retries
    seconds: float = 0.0


def run(ens, steps: int, *, transient: int = 0, stats_every: int = 10, checkpoint_every: int = 0,
        checkpoint_path: Optional[str] = None, log_path: Optional[str] = None, retry_factor: float = 0.5,
        max_retries: int = 2) -> RunReport:
    """Advance `ens` (a paper_2506_23712_gb300.ens.Ensemble or anything with
    the same methods) by `steps` steps.  Statistics are accumulated every
    `stats_every` steps once `transient` steps are done.  With a checkpoint
    path the state is saved at the start and every `checkpoint_every` steps
    (0: only at the start), and non-finite members are recovered as described
    in the module docstring; without one a non-finite member stops the run.
    One JSON object per block of `stats_every` steps goes to `log_path`."""
    if steps < 0 or stats_every < 1 or transient < 0 or checkpoint_every < 0:
        raise ValueError("steps, transient, checkpoint_every >= 0 and stats_every >= 1")
    rep = RunReport()
    t0 = time.perf_counter()
    log = open(log_path, "a") if log_path else None
    rules = [(m.dt, m.cfl, m.dt_max) for m in ens.members]
    initial = list(rules)
    first_snapshot = True
    saved = {"step": 0, "snapshots": 0, "first": True}

    def save():
        ens.save(checkpoint_path)
        rep.checkpoints += 1
        saved.update(step=rep.steps_done, snapshots=rep.snapshots, first=first_snapshot)

    try:
        if checkpoint_path:
            save()
        while rep.steps_done < steps:
            n = min(stats_every, steps - rep.steps_done)
            ens.step(n)
            diags = ens.diagnostics(raise_on_flag=False)
            bad = [i for i, d in enumerate(diags) if d["flags"] & FLAG_NONFINITE]
            if bad:
                if not checkpoint_path:
                    rep.failed = bad
                    break
                exhausted = [i for i in bad if rep.retried.get(i, 0) >= max_retries]
                if exhausted:
                    rep.failed = exhausted
                    break
                ens.load(checkpoint_path)
                rep.rollbacks += 1
                rep.steps_done, rep.snapshots = saved["step"], saved["snapshots"]
                first_snapshot = saved["first"]
                for i in bad:
                    rep.retried[i] = rep.retried.get(i, 0) + 1
                    dt, cfl, dt_max = rules[i]
                    rules[i] = (dt * retry_factor, cfl, dt_max) if dt > 0 else (dt, cfl * retry_factor, dt_max)
                # the checkpoint holds the time-step rules of its own time:
                # re-apply every rule changed since the start
                for i, r in enumerate(rules):
                    if r != initial[i]:
                        ens.set_timestep(i, *r)
                if log:
                    log.write(json.dumps({"event": "rollback", "to_step": rep.steps_done, "members": bad,
                                          "rules": {i: rules[i] for i in bad}}) + "\n")
                continue
            rep.steps_done += n
            if rep.steps_done > transient:
                ens.gradient_stats(accumulate=not first_snapshot)
                first_snapshot = False
                rep.snapshots += 1
            if log:
                log.write(json.dumps({"step": rep.steps_done, "snapshots": rep.snapshots,
                                      "diagnostics": diags}) + "\n")
            if checkpoint_path and checkpoint_every and rep.steps_done % checkpoint_every == 0:
                save()
    finally:
        if log:
            log.close()
        rep.seconds = time.perf_counter() - t0
    return rep
