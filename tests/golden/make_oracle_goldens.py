"""Writes the stored oracle values that the large GPU parity tests compare
against.  Calls only ``oracle/`` (the FP64 CPU oracle) and the seeded input
module ``ens_inputs``; nothing here touches the CUDA library.

Three kinds of files, all numpy ``.npz`` beside this script:

* ``one_step_<N>.npz``: one IF-RK3 step (CFL 0.2, Sec. IV) of members at the
  grid sizes whose oracle step takes minutes (256, 384, 512), from the seeded
  initial field; stored for a fixed sample of modes (every kept mode with
  max_i |k_i| <= 3, every forcing-band mode, 2048 seeded random kept modes,
  all three components), with the step's dt, E, dissipation and injected
  power, and the oracle's gradient statistics of the stepped field (joint Q-R,
  dissipation and enstrophy histograms, moments).  The GPU tests compare
  their own field on the same sample (relative L2, Sec. IV tolerances) and
  their statistics of their own field under the 2% rule.
* ``ten_steps_256.npz``: ten IF-RK3 steps (CFL 0.2) of the central member
  of the 64 x 256^3 benchmark ensemble, stored on the same kind of mode
  sample, with the diagnostics after every step.
* ``ensemble_64_long_run.npz``: the 16-member 64^3 ensemble (nu 0.01, band
  [3, 5], lambda on a uniform grid over [-3, 3], IF-RK3, CFL 0.2 capped at
  0.01) run 1000 steps; gradient statistics accumulated every 10 steps after
  step 500 (time averages over the second half of the run, Sec. IV), and the
  energy, dissipation and time at steps 500 and 1000.

Run from the repository root:
    python tests/golden/make_oracle_goldens.py one_step 256 384 512
    python tests/golden/make_oracle_goldens.py ten_steps
    python tests/golden/make_oracle_goldens.py long_run [--jobs 4]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import ens_inputs as I  # noqa: E402
import oracle as O  # noqa: E402

KEYS = ("N", "nu", "lam", "eps_bar", "k_lo", "k_hi", "dt", "cfl", "dt_max", "rk_order", "seed", "init_energy")

# histogram layout of the stored statistics (64 x 64 joint bins, 256-bin
# tails over [-8, 8) decades, units from eps_norm = 0.1 and the member nu)
HIST = dict(qr_bins=64, q_lim=10.0, r_lim=10.0, tail_bins=256, tail_lo=-8.0, tail_hi=8.0, eps_norm=0.1)

LONG_STEPS = 1000
LONG_FIRST = 500      # statistics after this step ...
LONG_EVERY = 10       # ... every this many steps


def oracle_member(d):
    return O.Member(**{k: d[k] for k in KEYS})


def one_step_cases(N):
    """Members of the workloads that use grid size N (names of ens_inputs)."""
    if N == 256:
        ds = I.ensemble_256()
        lams = np.array([d["lam"] for d in ds])
        return [("ensemble_256[%d]" % i, ds[i]) for i in (int(np.argmin(np.abs(lams))), int(np.argmax(lams)))]
    if N == 384:
        ds = [d for d in I.uneven_batch() if d["N"] == 384]
        return [("uneven_batch 384[0]", ds[0]), ("uneven_batch 384[3]", ds[-1])]
    if N == 512:
        ds = I.mixed_resolution()
        hi = [i for i, d in enumerate(ds) if d["N"] == 512]
        top = max(hi, key=lambda i: ds[i]["lam"])
        return [("mixed_resolution[%d]" % top, ds[top]), ("reference_512", I.reference_512()[0])]
    raise SystemExit("no one-step case for N=%d" % N)


def mode_sample(N, k_lo, k_hi, seed):
    """(kx index, ky index, kz) of the sampled kept modes, deduplicated."""
    kc = O.kc(N)
    k = np.fft.fftfreq(N, 1.0 / N).astype(np.int64)
    out = set()
    for ix in range(N):
        for iy in range(N):
            kx, ky = int(k[ix]), int(k[iy])
            if abs(kx) > kc or abs(ky) > kc:
                continue
            for kz in range(kc + 1):
                k2 = kx * kx + ky * ky + kz * kz
                low = max(abs(kx), abs(ky), kz) <= 3
                band = k_lo * k_lo - 1e-9 <= k2 <= k_hi * k_hi + 1e-9
                if low or band:
                    out.add((ix, iy, kz))
    rng = np.random.default_rng(seed)
    idx = np.concatenate([np.arange(0, kc + 1), np.arange(N - kc, N)])
    for _ in range(2048):
        out.add((int(rng.choice(idx)), int(rng.choice(idx)), int(rng.integers(0, kc + 1))))
    return np.array(sorted(out), dtype=np.int64)


def run_one_step(N):
    cases = one_step_cases(N)
    rec = {}
    for ci, (name, d) in enumerate(cases):
        t0 = time.time()
        m = oracle_member(d)
        uh = O.initial_field(m)
        st, diag = O.step(m, uh, 1)
        assert st == 0, (name, st)
        modes = mode_sample(N, d["k_lo"], d["k_hi"], seed=N + ci)
        vals = uh[:, modes[:, 0], modes[:, 1], modes[:, 2]]
        h = O.HistSpec(nu_norm=d["nu"], **HIST)
        counts, moments = O.gradient_stats(uh, d["nu"], h)
        rec["c%d_desc" % ci] = json.dumps(dict(d, name=name))
        rec["c%d_modes" % ci] = modes
        rec["c%d_values" % ci] = vals
        rec["c%d_diag" % ci] = np.array([diag[k] for k in ("t", "dt", "E", "diss", "EB", "P", "umax")])
        rec["c%d_counts" % ci] = counts
        rec["c%d_moments" % ci] = moments
        print("one_step N=%d %s: %.1f s, %d modes" % (N, name, time.time() - t0, len(modes)), flush=True)
    rec["cases"] = np.array(len(cases))
    rec["hist"] = json.dumps(HIST)
    path = os.path.join(HERE, "one_step_%d.npz" % N)
    np.savez_compressed(path, **rec)
    print("wrote", path)


def run_ten_steps():
    ds = I.ensemble_256()
    lams = np.array([d["lam"] for d in ds])
    i = int(np.argmin(np.abs(lams)))
    d = ds[i]
    m = oracle_member(d)
    uh = O.initial_field(m)
    keys = ("t", "dt", "E", "diss", "EB", "P", "umax")
    diags = []
    t = 0.0
    t0 = time.time()
    for s in range(10):
        st, diag = O.step(m, uh, 1, t)
        assert st == 0, (s, st)
        t = diag["t"]
        diags.append([diag[k] for k in keys])
    modes = mode_sample(d["N"], d["k_lo"], d["k_hi"], seed=2560)
    path = os.path.join(HERE, "ten_steps_256.npz")
    np.savez_compressed(path, desc=json.dumps(dict(d, name="ensemble_256[%d]" % i, index=i)), modes=modes,
                        values=uh[:, modes[:, 0], modes[:, 1], modes[:, 2]], diags=np.array(diags))
    print("wrote %s in %.0f s" % (path, time.time() - t0))


def long_run_member(i):
    d = I.ensemble_64()[i]
    m = oracle_member(d)
    uh = O.initial_field(m)
    h = O.HistSpec(nu_norm=d["nu"], **HIST)
    counts = np.zeros(h.counts_len, dtype=np.uint64)
    moments = np.zeros(O.NMOM, dtype=np.float64)
    t = 0.0
    diag_mid = None
    for s in range(1, LONG_STEPS + 1):
        st, diag = O.step(m, uh, 1, t)
        assert st == 0, (i, s, st)
        t = diag["t"]
        if s == LONG_FIRST:
            diag_mid = diag
        if s > LONG_FIRST and s % LONG_EVERY == 0:
            O.gradient_stats(uh, d["nu"], h, counts, moments)
    keys = ("t", "dt", "E", "diss", "EB", "P", "umax")
    return i, counts, moments, np.array([diag_mid[k] for k in keys]), np.array([diag[k] for k in keys])


def run_long(jobs):
    n = len(I.ensemble_64())
    t0 = time.time()
    if jobs > 1:
        import multiprocessing as mp
        os.environ.setdefault("OMP_NUM_THREADS", str(max(1, (os.cpu_count() or 1) // jobs)))
        with mp.get_context("spawn").Pool(jobs) as pool:
            res = pool.map(long_run_member, range(n))
    else:
        res = [long_run_member(i) for i in range(n)]
    res.sort(key=lambda r: r[0])
    path = os.path.join(HERE, "ensemble_64_long_run.npz")
    np.savez_compressed(path, counts=np.stack([r[1] for r in res]), moments=np.stack([r[2] for r in res]),
                        diag_mid=np.stack([r[3] for r in res]), diag_end=np.stack([r[4] for r in res]),
                        members=json.dumps(I.ensemble_64()), hist=json.dumps(HIST),
                        schedule=np.array([LONG_STEPS, LONG_FIRST, LONG_EVERY]))
    print("wrote %s in %.0f s" % (path, time.time() - t0))


def main():
    p = argparse.ArgumentParser()
    p.add_argument("what", choices=["one_step", "ten_steps", "long_run"])
    p.add_argument("sizes", nargs="*", type=int)
    p.add_argument("--jobs", type=int, default=1)
    a = p.parse_args()
    O.build()
    if a.what == "one_step":
        for N in a.sizes or [256, 384, 512]:
            run_one_step(N)
    elif a.what == "ten_steps":
        run_ten_steps()
    else:
        run_long(a.jobs)


if __name__ == "__main__":
    main()
