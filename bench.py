"""Benchmark of the ensemble DNS hot path on GB300.

Workload (one "step" = one IF-RK3 step of every member): 64 members on 256^3
grids, nu = 0.005, forcing band 6 <= |k| <= 8 at injection rate
exp(lambda) * 0.1 with lambda ~ N(0, 2^2) clipped to [-5.1, 5.8], CFL 0.2
(the shape of the paper's ens256 ensemble, Sec. IV, Table I).  Synthetic
seeded initial fields; the state (8.6 GB) is far larger than L2.

Prints one JSON line: member-steps/s (value), grid-point updates/s, the
roofline of the dominant kernel against the measured HBM copy bandwidth, the
FP64 CPU oracle on the host cores (cpu_baseline), the same metric through
the C ABI with the state streamed from/to pinned host memory every step
(e2e), SM clocks sampled during the timed region, and the plain
one-member-at-a-time torch.fft FP32 path on the same GPU for comparison.

--impl reference times the FP64 oracle (the reference arm) on the host cores
on a bounded sample of the same workload per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ensemble member-steps/s at 256^3, batched FP32 vs plain; % of HBM roofline"
UNIT = "member-steps/s"
WORKLOAD = "ensemble_256: 64 members x 256^3, nu=0.005, band 6<=|k|<=8, eps=exp(lambda)*0.1, " \
           "lambda~N(0,2^2) clipped [-5.1,5.8], IF-RK3, CFL 0.2"
PASS_NAMES = ["inv_x", "inv_y", "z_nonlinear", "fwd_y", "fwd_x_update"]
PASS_KERNELS = ["k_inv_x", "k_inv_y", "k_znl", "k_fwd_y", "k_fwd_x"]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--members", type=int, default=64)
    p.add_argument("--N", type=int, default=256)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-uneven", action="store_true")
    p.add_argument("--no-surrogate", action="store_true")
    p.add_argument("--no-tune", action="store_true", help="keep the default pass variants")
    p.add_argument("--no-mixed", action="store_true", help="skip the mixed-resolution / 512^3 measurements")
    p.add_argument("--set-tuning", default="", help="KEY=VAL,... applied to every grid-size group after "
                   "autotuning (for profiling a given variant), e.g. fx_split=1")
    return p.parse_args()


def parse_cpulist(text):
    cpus = set()
    for part in text.strip().split(","):
        if not part:
            continue
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        else:
            cpus.add(int(part))
    return cpus


def bind_host_to_gpu(local_rank):
    """Run this process on the CPU cores local to the GPU (sysfs local_cpulist
    of its PCI function), so that the page-locked buffers of the end-to-end
    measurement are allocated in the memory next to it.  Returns what was
    done, for the JSON line."""
    try:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        idx = vis.split(",")[local_rank] if vis else str(local_rank)
        out = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader", "-i", idx],
                             capture_output=True, text=True, timeout=30).stdout.strip().lower()
        dom, rest = out.split(":", 1)
        path = "/sys/bus/pci/devices/%04x:%s/local_cpulist" % (int(dom, 16), rest)
        with open(path) as f:
            cpus = parse_cpulist(f.read()) & os.sched_getaffinity(0)
        if not cpus:
            return {"bound": False, "why": "no local cores listed for " + out}
        os.sched_setaffinity(0, cpus)
        return {"bound": True, "pci": out, "cores": len(cpus)}
    except Exception as e:   # the measurement still runs, unbound
        return {"bound": False, "why": str(e)[:120]}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# plain one-member-at-a-time FP32 path (comparison baseline; torch.fft + unfused ops)
# ---------------------------------------------------------------------------
def plain_member_steps(member, nsteps, torch):
    N = member["N"]
    dev = "cuda"
    kc = (N + 2) // 3 - 1
    k = torch.fft.fftfreq(N, 1.0 / N, device=dev)
    kz = torch.arange(N // 2 + 1, device=dev, dtype=torch.float32)
    KX, KY, KZ = torch.meshgrid(k, k, kz, indexing="ij")
    K = torch.stack([KX, KY, KZ])
    k2 = (K * K).sum(0)
    k2s = torch.where(k2 == 0, torch.ones_like(k2), k2)
    mask = ((KX.abs() <= kc) & (KY.abs() <= kc) & (KZ <= kc)).to(torch.float32)
    band = ((k2 >= member["k_lo"] ** 2 - 1e-9) & (k2 <= member["k_hi"] ** 2 + 1e-9)).to(torch.float32)
    wgt = torch.where(KZ == 0, torch.ones_like(KZ), 2 * torch.ones_like(KZ))
    eps_inj = math.exp(member["lam"]) * member["eps_bar"]
    nu = member["nu"]
    g = torch.Generator(device=dev).manual_seed(member["seed"])
    u0 = torch.randn((3, N, N, N), device=dev, generator=g)
    uh = torch.fft.rfftn(u0, dim=(1, 2, 3), norm="forward") * mask
    uh = uh - K * (K * uh).sum(0) / k2s
    uh = uh * (0.5 / (0.5 * (wgt * (uh.abs() ** 2).sum(0)).sum())).sqrt()

    def rhs(v):
        w = 1j * torch.linalg.cross(K.to(v.dtype), v, dim=0)
        u = torch.fft.irfftn(v, s=(N, N, N), dim=(1, 2, 3), norm="forward")
        om = torch.fft.irfftn(w, s=(N, N, N), dim=(1, 2, 3), norm="forward")
        umax = u.abs().max()
        n = torch.linalg.cross(u, om, dim=0)
        nh = torch.fft.rfftn(n, dim=(1, 2, 3), norm="forward") * mask
        nh = nh - K * (K * nh).sum(0) / k2s
        EB = 0.5 * (band * wgt * (v.abs() ** 2).sum(0)).sum()
        return nh + (eps_inj / (2 * EB)) * band * v, umax

    def E(h):
        return torch.exp(-nu * k2 * h)

    for _ in range(nsteps):
        F, umax = rhs(uh)
        dt = member["cfl"] * (2 * math.pi / N) / umax
        u1 = E(dt) * (uh + dt * F)
        F1, _ = rhs(u1)
        u2 = 0.75 * E(dt / 2) * uh + 0.25 * E(-dt / 2) * (u1 + dt * F1)
        F2, _ = rhs(u2)
        uh = E(dt) * uh / 3 + 2.0 / 3.0 * E(dt / 2) * (u2 + dt * F2)
    return uh


def time_plain(members, torch, n_members=2, nsteps=2):
    torch.cuda.synchronize()
    plain_member_steps(members[0], 1, torch)   # warm-up (cuFFT plans)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    for m in members[:n_members]:
        plain_member_steps(m, nsteps, torch)
    end.record()
    torch.cuda.synchronize()
    sec = start.elapsed_time(end) / 1e3
    return n_members * nsteps / sec


# ---------------------------------------------------------------------------
# the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
def oracle_member(d):
    import oracle as O
    return O.Member(N=d["N"], nu=d["nu"], lam=d["lam"], eps_bar=d["eps_bar"], k_lo=d["k_lo"], k_hi=d["k_hi"],
                    dt=d["dt"], cfl=d["cfl"], dt_max=d["dt_max"], rk_order=d["rk_order"], seed=d["seed"],
                    init_energy=d["init_energy"])


ONE_CORE_SNIPPET = """
import sys, time, json
sys.path.insert(0, %r)
import oracle as O
m = O.Member(**json.loads(%r))
uh = O.initial_field(m)
t0 = time.perf_counter()
O.rhs(m, uh)
print(json.dumps({"sec": time.perf_counter() - t0}))
"""


def cpu_baseline(member_dict):
    """The FP64 oracle on the host cores: one full IF-RK3 step of one 256^3
    member on every core, and one right-hand-side evaluation (a third of a
    step) of the same member on one core, in a child process pinned to one
    core with one OpenMP thread."""
    import oracle as O
    O.build()
    m = oracle_member(member_dict)
    uh = O.initial_field(m)
    t0 = time.perf_counter()
    st, _ = O.step(m, uh, 1)
    sec = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", len(os.sched_getaffinity(0))))
    out = {"value": 1.0 / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "one IF-RK3 step of one %d^3 member (FP64 oracle, own FFT) on %d cores, %.1f s" % (
               m.N, cores, sec)}
    try:
        desc = {k: getattr(m, k) for k in ("N", "nu", "lam", "eps_bar", "k_lo", "k_hi", "dt", "cfl", "dt_max",
                                           "rk_order", "seed", "init_energy")}
        core = min(os.sched_getaffinity(0))
        r = subprocess.run([sys.executable, "-c", ONE_CORE_SNIPPET % (ROOT, json.dumps(desc))],
                           env=dict(os.environ, OMP_NUM_THREADS="1"), capture_output=True, text=True, timeout=300,
                           preexec_fn=lambda: os.sched_setaffinity(0, {core}))
        sec1 = json.loads(r.stdout.strip().splitlines()[-1])["sec"]
        out["single_core"] = {"value": (1.0 / 3.0) / sec1, "unit": UNIT, "cores": 1, "kind": "oracle",
                              "sample": "one right-hand-side evaluation (a third of an IF-RK3 step) of one "
                                        "%d^3 member on 1 core, %.1f s" % (m.N, sec1)}
    except Exception as e:   # the all-core figure stands on its own
        out["single_core"] = {"value": None, "why": str(e)[:160]}
    return out


def run_reference(args, members):
    """Reference arm: the FP64 oracle, each step = one right-hand-side
    evaluation (one RK stage, 1/3 of a member-step) of one 256^3 member."""
    import oracle as O
    O.build()
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    m = oracle_member(members[0])
    uh = O.initial_field(m)
    for _ in range(args.warmup):
        O.rhs(m, uh)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.rhs(m, uh)
    sec = time.perf_counter() - t0
    value = (args.steps / 3.0) / sec
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = "per step: one right-hand-side evaluation (one of three RK3 stages) of one %d^3 member" % m.N
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "members": len(members), "N": m.N},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def hellinger(p, q):
    p = np.asarray(p, dtype=np.float64).ravel()
    q = np.asarray(q, dtype=np.float64).ravel()
    p, q = p / p.sum(), q / q.sum()
    return float(np.sqrt(max(0.0, 1.0 - np.sum(np.sqrt(p * q)))))


def measure_surrogate(E, ens, descs, torch, steps=800):
    """Learned lambda interpolant on this ensemble's own histograms: training
    throughput, the tcgen05 hidden-layer GEMM against the BF16 peak, and the
    512-point quadrature mixture against the member quadrature (Hellinger)."""
    ens.gradient_stats(accumulate=False)
    counts, _ = ens.stats()
    h = ens.hist
    lams = np.array([d.lam for d in descs])
    per = h.qr_bins ** 2 + 2 * h.tail_bins
    S = E.Surrogate(seed=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = S.train(lams, counts, h, steps, lr=4e-3)
    t_train = time.perf_counter() - t0
    rows_q = 512 * per
    gemm_ms = S.time_gemm(rows_q, iters=5)
    gemm_tflops = 2.0 * pad128(rows_q) * 256 * 256 / (gemm_ms / 1e3) / 1e12
    # fused inference (features -> 3 tcgen05 layers -> head) over the 512-point quadrature
    infer_ms = S.time_infer(h, 512, iters=5)
    infer_flops = 2.0 * rows_q * (64 * 256 + 2 * 256 * 256 + 256)
    tflops = infer_flops / (infer_ms / 1e3) / 1e12
    Z = 1.5 * math.log(261.0 / 63.0)
    s = np.sort(np.unique(lams))
    lo, hi = s[0] - 0.5 * (s[1] - s[0]), s[-1] + 0.5 * (s[-1] - s[-2])
    ref = E.ens_mixture(ens.ctx, len(lams), h, kind=E.W_GAUSS_PAPER, c=0.023, Z=Z)
    t0 = time.perf_counter()
    sur = S.mixture(h, lo, hi, 512, kind=E.W_GAUSS_PAPER, c=0.023, Z=Z)
    t_inf = time.perf_counter() - t0
    S.close()
    gain = held_out_gain(E, lams, counts, h, steps)
    peak = measured_bf16()
    return {"members": len(lams), "bins_per_member": per, "train_steps": steps, "train_s": t_train,
            "held_out_gain": gain,
            "train_rows_per_step": len(lams) * per, "final_loss": loss,
            "quadrature_points": 512, "mixture_s": t_inf,
            "hellinger_vs_member_quadrature": {k: hellinger(sur[k], ref[k]) for k in ("pdf_qr", "pdf_eps", "pdf_ens")},
            "Z": Z, "roofline": {"bound": "tensor", "kernel": "k_mlp_infer_pair", "achieved": tflops, "peak": peak[0],
                                  "unit": "TFLOP/s", "frac": tflops / peak[0], "peak_source": peak[1],
                                  "rows": rows_q, "flops_per_launch": infer_flops, "ms": infer_ms},
            "layer_gemm": {"kernel": "k_gemm_tc<256>", "shape": "%d x 256 x 256 BF16 -> FP32" % pad128(rows_q),
                           "ms": gemm_ms, "TFLOPs": gemm_tflops,
                           "note": "training-path layer GEMM; FP32 output makes it HBM-bound (86 flop/B)"}}


def held_out_gain(E, lams, counts, h, steps):
    """What the interpolant gains over the method without it: trained on
    every other member in lambda order, evaluated at the held-out interior
    members against the nearest simulated member and against linear
    interpolation in lambda (mean Hellinger over held-out members, per PDF)."""
    nq, nt = h.qr_bins, h.tail_bins
    order = np.argsort(lams)
    lam_s, cnt_s = lams[order], counts[order]
    parts = [slice(0, nq * nq), slice(nq * nq, nq * nq + nt), slice(nq * nq + nt, nq * nq + 2 * nt)]

    def norm(c):
        c = np.asarray(c, dtype=np.float64)
        return np.concatenate([c[x] / max(c[x].sum(), 1.0) for x in parts])
    P = np.array([norm(c) for c in cnt_s])
    ev = np.arange(0, len(lam_s), 2)
    od = np.arange(1, len(lam_s) - 1, 2)
    if len(od) == 0:
        return {"note": "fewer than three members: no held-out member"}
    S = E.Surrogate(seed=5)
    S.train(lam_s[ev], cnt_s[ev], h, steps, lr=4e-3)
    q = S.density(lam_s[od], h)
    S.close()
    res = {"surrogate": [], "nearest_member": [], "linear_in_lambda": []}
    for j, i in enumerate(od):
        near = i - 1 if lam_s[i] - lam_s[i - 1] <= lam_s[i + 1] - lam_s[i] else i + 1
        a = (lam_s[i + 1] - lam_s[i]) / max(lam_s[i + 1] - lam_s[i - 1], 1e-12)
        lin = a * P[i - 1] + (1 - a) * P[i + 1]
        for key, est in (("surrogate", q[j]), ("nearest_member", P[near]), ("linear_in_lambda", lin)):
            res[key].append([hellinger(est[x], P[i][x]) for x in parts])
    out = {k: dict(zip(("pdf_qr", "pdf_eps", "pdf_ens"), np.mean(v, axis=0).round(5).tolist()))
           for k, v in res.items()}
    means = {k: float(np.mean(v)) for k, v in res.items()}
    out["best"] = min(means, key=means.get)
    out["note"] = ("trained on every other member in lambda order, evaluated at the %d held-out interior members "
                   "(single snapshot of the benchmark ensemble)" % len(od))
    return out


def pad128(r):
    return (r + 127) // 128 * 128


def measured_bf16():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "measured bf16_tflops (burst cuBLAS)"
    return 1900.0, "fallback"


def measure_uneven(E, torch, steps=3, tune=True):
    """Uneven-size batch (24 x 128^3, 12 x 256^3, 4 x 384^3): all members in
    one graph per step (one branch per grid size) vs member-by-member
    launches of the same kernels."""
    import ens_inputs as I
    ms = [E.Member(N=d["N"], nu=d["nu"], lam=d["lam"], eps_bar=d["eps_bar"], k_lo=d["k_lo"], k_hi=d["k_hi"],
                   dt=d["dt"], cfl=d["cfl"], dt_max=d["dt_max"], rk_order=d["rk_order"], seed=d["seed"],
                   init_energy=d["init_energy"]) for d in I.uneven_batch()]
    stream = torch.cuda.current_stream()
    ens = E.Ensemble(ms, hist=E.hist_spec(nu_norm=ms[0].nu), stream=stream)
    out = {"workload": "24 x 128^3 + 12 x 256^3 + 4 x 384^3, IF-RK3, CFL 0.2, k_max eta >= 1.5",
           "members": len(ms), "steps": steps}
    if tune:
        out["tuning"] = ens.autotune(steps=2)
    tuned = ens.tuning()

    def with_persistent(flag):
        t = json.loads(json.dumps(tuned))
        t["persistent"] = flag
        ens.set_tuning(t)
    # the autotuner's choice, then each design on its own: all members in one
    # persistent launch per RK stage, the graph of per-pass launches (one
    # branch or chain per grid size), and member-by-member launches
    for mode in ("batched", "persistent", "graph_branches", "sequential"):
        if mode == "persistent":
            with_persistent(1)
        elif mode == "graph_branches":
            with_persistent(0)
        run = (lambda k: E.ens_step_sequential(ens.ctx, k)) if mode == "sequential" else (lambda k: ens.step(k))
        run(1)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run(steps)
        b.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) / 1e3
        out[mode] = {"member_steps_per_s": len(ms) * steps / sec, "ms_per_step": 1e3 * sec / steps}
    out["batched_over_sequential"] = out["batched"]["member_steps_per_s"] / out["sequential"]["member_steps_per_s"]
    out["persistent_over_graph_branches"] = (out["persistent"]["member_steps_per_s"] /
                                             out["graph_branches"]["member_steps_per_s"])
    flags = sum(1 for d in ens.diagnostics(raise_on_flag=False) if d["flags"])
    out["flagged_members"] = flags
    ens.close()
    return out


def measure_mixed(E, torch, steps=3, tune=True):
    """Mixed-resolution ensemble (the 64 x 256^3 members, those at lambda >=
    3.2 on 512^3 grids) and the single 512^3 reference-run shape, each timed
    over a few graph replays after one untimed step."""
    import ens_inputs as I

    def mk(ds):
        return [E.Member(N=d["N"], nu=d["nu"], lam=d["lam"], eps_bar=d["eps_bar"], k_lo=d["k_lo"],
                         k_hi=d["k_hi"], dt=d["dt"], cfl=d["cfl"], dt_max=d["dt_max"], rk_order=d["rk_order"],
                         seed=d["seed"], init_energy=d["init_energy"]) for d in ds]
    stream = torch.cuda.current_stream()
    out = {}
    for name, ds in (("mixed_resolution", I.mixed_resolution()), ("reference_512", I.reference_512())):
        ms = mk(ds)
        ens = E.Ensemble(ms, hist=E.hist_spec(nu_norm=ms[0].nu), stream=stream)
        rec = {"members": len(ms), "grids": {str(n): sum(1 for m in ms if m.N == n) for n in sorted({m.N for m in ms})}}
        if tune:
            rec["tuning"] = ens.autotune(steps=2)
        ens.step(1)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ens.step(steps)
        b.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) / 1e3
        pts = sum(m.N ** 3 for m in ms)
        rec.update(steps=steps, ms_per_step=1e3 * sec / steps, member_steps_per_s=len(ms) * steps / sec,
                   grid_point_updates_per_s=pts * steps / sec,
                   flagged_members=sum(1 for d in ens.diagnostics(raise_on_flag=False) if d["flags"]))
        ens.close()
        out[name] = rec
    out["reference_512"]["note"] = ("throughput of the reference-run shape only: a statistically "
                                    "stationary 512^3 reference needs ~10^5 steps")
    return out


def traffic_for(kernel):
    """ncu DRAM bytes per launch of the kernel (profiles/traffic.json), or None
    if the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        t = json.load(f)
    if t.get("source_sha256") != pass_sources_sha256():
        return None
    return t.get("kernels", {}).get(kernel)


# the files that define the RK-stage pass kernels (their counters go stale
# when any of these changes; the statistics pass is not among them)
PASS_SOURCES = ["ens_fft.cuh", "ens_fxsplit.cuh", "ens_internal.h", "ens_kernels.cuh", "ens_sized.cu", "ens_tma.cuh",
                "ens_znl.cuh"]


def pass_sources_sha256():
    src = os.path.join(ROOT, "paper_2506_23712_gb300", "csrc")
    h = hashlib.sha256()
    for name in PASS_SOURCES:
        with open(os.path.join(src, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def main():
    args = parse()
    import ens_inputs as I
    members = I.ensemble_256(args.members, args.N)
    if args.impl == "reference":
        run_reference(args, members)
        return

    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2506_23712_gb300 import ens as E

    # weak scaling: every rank advances its own ensemble of the same shape
    descs = [E.Member(N=d["N"], nu=d["nu"], lam=d["lam"], eps_bar=d["eps_bar"], k_lo=d["k_lo"], k_hi=d["k_hi"],
                      dt=d["dt"], cfl=d["cfl"], dt_max=d["dt_max"], rk_order=d["rk_order"],
                      seed=d["seed"] + 100000 * rank, init_energy=d["init_energy"]) for d in members]
    hist = E.hist_spec(nu_norm=0.005, eps_norm=0.1)
    stream = torch.cuda.current_stream()
    ens = E.Ensemble(descs, hist=hist, stream=stream)
    n_mem = len(descs)
    # pass variants picked by the library's autotuner on these members (the
    # member state is restored afterwards; untimed)
    tuning = None if args.no_tune else ens.autotune(steps=2)
    if args.set_tuning:
        t = ens.tuning()
        for kv in args.set_tuning.split(","):
            k, v = kv.split("=")
            for g in t["groups"]:
                g[k.strip()] = int(v)
        ens.set_tuning(t)
        tuning = dict(ens.tuning(), forced=args.set_tuning)
    kps = E.ens_kernels_per_step(ens.ctx)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        ens.step(1)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    ens.step(args.steps)
    end.record(stream)
    barrier()
    clk = clocks.stop()
    ms = start.elapsed_time(end)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_per_step = ms / args.steps
    value = world * n_mem * args.steps / (ms / 1e3)
    diags = ens.diagnostics(raise_on_flag=False)
    flagged = sum(1 for d in diags if d["flags"])

    # per-pass device times (CUDA events on the library's stream), stage 1
    hbm, peak_kind = measured_peaks()
    passes = {}
    reps = 5
    for p, name in enumerate(PASS_NAMES):
        E.ens_run_pass(ens.ctx, p, 1)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            E.ens_run_pass(ens.ctx, p, 1)
        b.record(stream)
        torch.cuda.synchronize()
        pms = a.elapsed_time(b) / reps
        nbytes = E.ens_pass_bytes(ens.ctx, p, 1)
        passes[name] = {"ms": round(pms, 4), "algorithmic_GB": round(nbytes / 1e9, 4),
                        "GBps": round(nbytes / 1e9 / (pms / 1e3), 1),
                        "frac": round(nbytes / 1e9 / (pms / 1e3) / hbm, 4)}
    # statistics snapshot (gradient fields, invariants, histograms, moments of
    # every member) and the FP64 lambda mixture of the snapshot
    ens.gradient_stats(accumulate=False)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(3):
        ens.gradient_stats(accumulate=False)
    b.record(stream)
    torch.cuda.synchronize()
    sms = a.elapsed_time(b) / 3
    sbytes = E.ens_pass_bytes(ens.ctx, 5, 0)
    t0 = time.perf_counter()
    E.ens_mixture(ens.ctx, n_mem, ens.hist, kind=E.W_GAUSS_PAPER, c=0.023, Z=1.5 * math.log(261.0 / 63.0))
    mix_ms = (time.perf_counter() - t0) * 1e3
    stats = {"ms": round(sms, 4), "algorithmic_GB": round(sbytes / 1e9, 4),
             "GBps": round(sbytes / 1e9 / (sms / 1e3), 1), "frac": round(sbytes / 1e9 / (sms / 1e3) / hbm, 4),
             "members": n_mem, "mixture_ms": round(mix_ms, 3),
             "note": "one ens_gradient_stats snapshot of all members (CUDA events); mixture: ens_mixture "
                     "with the paper's Gaussian lambda weights, host wall time incl. the copies"}
    dom = max(passes, key=lambda k: passes[k]["ms"])
    dom_idx = PASS_NAMES.index(dom)
    achieved = passes[dom]["GBps"]
    kernel = PASS_KERNELS[dom_idx]
    if kernel == "k_znl" and tuning and tuning["groups"][0]["z_variant"] == 1:
        kernel = "k_z"   # the row-group z-pass variant won the autotuning
    roofline = {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": round(achieved / hbm, 4), "peak_source": peak_kind + " hbm_gbs (copy)",
                "traffic": traffic_for(kernel),
                "algorithmic_bytes_per_launch": passes[dom]["algorithmic_GB"] * 1e9}
    step_bytes = sum(E.ens_pass_bytes(ens.ctx, p, s) for p in range(5) for s in range(3))
    step_frac = step_bytes / 1e9 / (ms_per_step / 1e3) / hbm

    # e2e: the state streamed from pinned host memory through the C ABI every step
    e2e = None
    if not args.no_e2e:
        nbytes = ens.state_bytes()
        all_cores = os.sched_getaffinity(0)
        numa = bind_host_to_gpu(local)
        host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        E.ens_get_state(ens.ctx, host.data_ptr(), nbytes)
        e2e_steps = max(2, min(args.steps, 5))
        E.ens_step_host(ens.ctx, host.data_ptr(), host.data_ptr(), nbytes, 0)   # creates the copy streams
        # three windows of e2e_steps steps; the host memory is shared with
        # other jobs on the machine, so the median window is reported
        windows = []
        for _w in range(3):
            barrier()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                E.ens_step_host(ens.ctx, host.data_ptr(), host.data_ptr(), nbytes, 0)
                dg, _ = E.ens_diagnostics(ens.ctx, n_mem, raise_on_flag=False)
            barrier()
            windows.append(time.perf_counter() - t0)
        sec = statistics.median(windows)
        # the same without overlap: upload, graph step, download one after another
        t1 = time.perf_counter()
        for _ in range(2):
            E.ens_set_state(ens.ctx, host.data_ptr(), nbytes)
            ens.step(1)
            E.ens_get_state(ens.ctx, host.data_ptr(), nbytes)
            E.ens_diagnostics(ens.ctx, n_mem, raise_on_flag=False)
        serial = world * n_mem * 2 / (time.perf_counter() - t1)
        # the copy rates seen by this buffer
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        E.ens_set_state(ens.ctx, host.data_ptr(), nbytes)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        E.ens_get_state(ens.ctx, host.data_ptr(), nbytes)
        t4 = time.perf_counter()
        numa.update(h2d_GBs=round(nbytes / (t3 - t2) / 1e9, 1), d2h_GBs=round(nbytes / (t4 - t3) / 1e9, 1))
        del host
        os.sched_setaffinity(0, all_cores)   # the CPU baseline below uses every core
        diag_bytes = n_mem * 96
        e2e = {"value": world * n_mem * e2e_steps / sec, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes + diag_bytes, "steps": e2e_steps,
               "windows_member_steps_per_s": [round(world * n_mem * e2e_steps / w, 1) for w in windows],
               "path": "ens_step_host(pinned host in/out, members in chunks tapered by a factor 3 at both ends: upload, step and download "
                       "overlapped) + ens_diagnostics", "serial_value": serial, "host_binding": numa}

    plain = None
    if not args.no_plain and rank == 0:
        pv = time_plain(members, torch)
        plain = {"value": pv, "unit": UNIT, "path": "one member at a time, torch.fft (cuFFT) FP32 + unfused torch ops",
                 "batched_over_plain": value / world / pv}
    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        cpu = cpu_baseline(members[0])

    surrogate = None
    if not args.no_surrogate and rank == 0:
        surrogate = measure_surrogate(E, ens, descs, torch)
    state_gb = ens.state_bytes() / 1e9
    ens.close()
    uneven = None
    if not args.no_uneven and rank == 0:
        uneven = measure_uneven(E, torch, tune=not args.no_tune)
    mixed = None
    if not args.no_mixed and rank == 0:
        mixed = measure_mixed(E, torch, tune=not args.no_tune)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "members": n_mem, "N": args.N, "rk_order": 3,
                           "grid_point_updates_per_s": value * args.N ** 3,
                           "l2": "inputs larger than L2 (state %.1f GB + pass buffers, %.0f GB of algorithmic "
                                 "HBM traffic per step)" % (state_gb, step_bytes / 1e9),
                           "parallelism": "replicas per GPU" if world > 1 else "single GPU",
                           "step_hbm_roofline_frac": round(step_frac, 4),
                           "tuning": tuning,
                           "flagged_members": flagged},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": kps * args.steps,
                "clocks": clk, "plain": plain, "passes": passes, "stats_snapshot": stats, "uneven_batch": uneven, "mixed_resolution": mixed,
                "surrogate": surrogate}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
