#!/usr/bin/env python
"""Benchmark of the fused MPCD collision interval on GB300.

Metric: MPCD solvent particle-steps/s (one particle-step = one solvent particle
advanced through one full collision interval: near-colloid MD sub-steps or free
flight, grid shift, sort, collision, reactions), mixed FP32 path, with the FP64
path on the same workload for comparison, and the HBM roofline fraction of the
dominant kernel.

Default workload: the batched ensemble of 256 independent replicas in one
launch per kernel (cube sides drawn from {16, 20, 24, 32, 40, 48}, density 10,
104,070,400 solvent in all), each holding one rigid Janus particle of 100-300
beads with a catalytic hemisphere, alpha = 130 deg, tau = 0.5, 25 MD sub-steps
of dt = 0.02 per collision: the mixed-FP32 batched MPCD step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload batch256|dimer32|sphere16|poiseuille128|thermal]
                    [--precision mixed|fp64]

With torchrun (N > 1) every rank runs an independent replica of the workload
(replicas only: the method has no data exchange between independent systems).
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MPCD solvent particle-steps/s, mixed-FP32 vs FP64 on 1 GB300; HBM roofline %"
UNIT = "particle-steps/s"
# algorithmic bytes per particle-step of the cell pass: record read + write
# (28 B mixed / 52 B fp64 of state each way) + bucket entry write + read
ALG_BYTES = {"mixed": 64, "fp64": 112}
L2_FLUSH_BYTES = 256 << 20
KERNEL_NAMES = {"cellpass": "k_cellpass", "md": "k_md", "prime": "k_particles", "obs": "k_obs_reduce"}
# sources that decide a kernel's memory traffic: the kernel, the shared
# headers and the host code that sizes its buffers and launch
KERNEL_SOURCES = {"k_cellpass": ["rmpcd_common.cuh", "rmpcd_kernels.cuh", "k_cellpass.cu", "capi.cu"]}


def workload(name, precision, seed_offset=0, n_replicas=None):
    """The workload as a list of replicas (cfg, colloids, bonds, body) and a description.
    n_replicas keeps the first replicas of the batched ensemble only (a smaller
    case of the same kernels, for profiling)."""
    from paper_1608_04904_gb300 import synth
    if name == "dimer32":
        reps = [synth.dimer32(precision=precision, seed=2 + seed_offset)]
        desc = ("reactive sphere dimer (C+N, sigma 2, M 100, bond 4.5), 32^3 periodic box, rho 10, "
                "327680 solvent, 50 MD sub-steps dt 0.01, alpha 90 deg, tau 0.5, kT 1/3, p_cat 1, bulk k 0.01")
    elif name == "dimer64":
        reps = [synth.dimer32(precision=precision, seed=2 + seed_offset, L=64)]
        desc = ("reactive sphere dimer as dimer32 in a 64^3 periodic box, rho 10, 2621440 solvent "
                "(larger than L2; profiling case)")
    elif name == "sphere16":
        reps = [synth.sphere16(precision=precision, seed=1 + seed_offset)]
        desc = "one WCA sphere (sigma 2, M 200), 16^3 periodic box, rho 10, 40960 solvent, 50 MD sub-steps"
    elif name == "poiseuille128":
        reps = [synth.poiseuille(precision=precision, seed=3 + seed_offset)]
        desc = ("Poiseuille channel 128^3 with stick walls in z, rho 10, 20971520 solvent, g 0.001 x, "
                "alpha 130 deg, tau 1")
    elif name == "thermal":
        reps = [synth.thermal(precision=precision, seed=5 + seed_offset)]
        desc = ("thermal-gradient suspension 256x64x64, rho 10, 10485760 solvent, 64 WCA spheres (sigma 2.5, "
                "M 150), colloid LJ eps 1 sigma 5.5 cut 2.5 sigma, MPC-AT slabs [0,8) kT 1.2 and [128,136) kT 0.8, "
                "50 MD sub-steps dt 0.01")
    elif name == "batch256":
        sides = synth.batch_sides(256, seed=4)[:n_replicas]
        reps = []
        for r, L in enumerate(sides):
            cfg, body = synth.batch_janus(L, seed=4 + r + 1000 * seed_offset, precision=precision)
            reps.append((cfg, [], [], body))
        desc = (f"{len(sides)} independent replicas in one launch per kernel, cube sides drawn from {{16,20,24,32,40,48}} "
                "(seed 4), rho 10, one rigid Janus particle each (100-300 beads on a sphere of radius 4, "
                "sigma_b 1, catalytic hemisphere A->B), alpha 130 deg, tau 0.5, 25 MD sub-steps dt 0.02")
        return reps, desc
    elif name == "network64":
        sides = synth.batch_sides(256, seed=4)[:64][:n_replicas]
        reps = []
        for r, L in enumerate(sides):
            cfg, body = synth.batch_janus(L, seed=4 + r + 1000 * seed_offset, precision="fp64")
            body = dict(body, network=synth.janus_network(body))
            reps.append((cfg, [], [], body))
        desc = (f"{len(sides)} independent replicas (the first of batch256: same sides, seeds and solvent), each "
                "Janus particle a bead network held by iterative RATTLE (links to each bead's ring of neighbours, "
                "edge-coloured; tolerance 1e-12) instead of a rigid body; FP64 (the network integrator's "
                "precision), 25 MD sub-steps dt 0.02")
        return reps, desc
    else:
        raise SystemExit(f"unknown workload {name}")
    return [(cfg, col, bonds, None) for cfg, col, bonds in reps], desc


def initial_state(rep):
    """Seeded solvent of one replica, outside its colloids or body."""
    from paper_1608_04904_gb300 import synth
    cfg, col, bonds, body = rep
    excl = col if body is None else synth.body_exclusion(body)
    return synth.solvent(cfg, excl, seed=cfg["seed"] + 100)


class _NetworkOracle:
    """The oracle's interval of a bead-network replica followed by its
    collision step (the same sequence a GPU interval runs)."""

    def __init__(self, oracle, cfg, state, net):
        import numpy as np
        from paper_1608_04904_gb300 import network
        x, v, fl = state
        links, d = net["links"], np.asarray(net["d"])
        order = network.order_by_color(links, network.color_links(links, len(net["xb"])))
        self.orc = oracle
        self.net = oracle.Network(net["xb"], net["vb"], net["mb"], net["eps_A"], net["eps_B"], net["catalytic"],
                                  net["sigma"], [links[k] for k in order], d[order])
        self.o = oracle.OracleSystem(cfg, x, v, fl, cell_order=CELL_ORDER)
        self.cfg = cfg

    def step(self, k):
        o = self.o
        for _ in range(k):
            rc, _ = self.orc.interval_network(self.cfg, o.x, o.v, o.flags, o.id, self.net, step=o.step_index)
            if rc != 0:
                raise RuntimeError(f"oracle network interval status {rc}")
            o.shift_and_sort()
            o.collide()
            o.react()
            o.step_index += 1


def oracle_system(oracle, rep, state):
    from paper_1608_04904_gb300 import synth
    cfg, col, bonds, body = rep
    x, v, fl = state
    if body is not None and "network" in body:
        return _NetworkOracle(oracle, cfg, state, body["network"])
    return oracle.OracleSystem(cfg, x, v, fl, colloids=synth.colloid_arrays(col) if col else None, bonds=bonds,
                               body=body, cell_order=CELL_ORDER)


def kernel_hash(kernel="k_cellpass"):
    h = hashlib.sha256()
    for s in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_1608_04904_gb300", "csrc", s), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(kernel, workload_name, precision, n_particles, cell_order="linear"):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or None
    when absent or taken on a different kernel build.  An entry captured on a
    smaller case of the same workload (bytes_per_particle) is scaled to the
    launch by its particle count: the traffic of the cell pass grows in
    proportion to the particles it moves."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if kernel not in KERNEL_SOURCES or d.get("kernel_hash") != kernel_hash(kernel):
        return None
    key = f"{kernel}/{workload_name}/{precision}" + ("" if cell_order == "linear" else f"/{cell_order}")
    e = d.get("kernels", {}).get(key)
    if e is None:
        return None
    if "bytes_per_particle" in e:
        return int(round(e["bytes_per_particle"] * n_particles))
    return e.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"rmpcd_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_throughput(ms, n_local, steps, device=None):
    """Whole-job particle-steps/s and the job's time in ms: every rank's
    particles (independent replicas, weak scaling) over the slowest rank's
    time.  Without an initialised process group of more than one rank, the
    local values."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        tm = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        tn = torch.tensor([float(n_local)], dtype=torch.float64, device=device)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        dist.all_reduce(tn, op=dist.ReduceOp.SUM)
        ms, n_all = float(tm.item()), float(tn.item())
    else:
        n_all = float(n_local)
    return n_all * steps / (ms / 1e3), ms


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                             timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample(name, precision, max_particles=2_000_000):
    """The replicas the CPU legs time: the workload itself, or for a batch its
    first replicas up to about max_particles solvent (at least one)."""
    reps, desc = workload(name, precision)
    out, n = [], 0
    for r in reps:
        st = initial_state(r)
        if out and n + len(st[0]) > max_particles:
            break
        out.append((r, st))
        n += len(st[0])
    return out, n, len(reps), desc


def time_oracle(oracle, sample, threads, budget_s, warmup=1, max_steps=10000):
    """Full collision intervals of every sampled replica on `threads` OpenMP
    threads until the budget is spent; returns (particle-steps/s, intervals, s)."""
    used = oracle.set_threads(threads)
    try:
        systems = [oracle_system(oracle, r, st) for r, st in sample]
        n = sum(len(st[0]) for _, st in sample)
        for _ in range(warmup):
            for o in systems:
                o.step(1)
        t0 = time.perf_counter()
        k = 0
        while True:
            for o in systems:
                o.step(1)
            k += 1
            el = time.perf_counter() - t0
            if (el >= budget_s and k >= 2) or k >= max_steps:
                break
    finally:
        oracle.set_threads(1)
    return n * k / el, k, el, used


def cpu_baseline(name, precision, budget_s=10.0):
    """The oracle, as it stands, on the host cores, on one thread and on every
    core (its OpenMP loops; results do not depend on the thread count): full
    collision intervals of a bounded sample of the same workload."""
    from oracle import oracle
    oracle.build()
    sample, n, n_rep, _ = oracle_sample(name, precision)
    v1, k1, e1, _ = time_oracle(oracle, sample, 1, budget_s)
    va, ka, ea, cores = time_oracle(oracle, sample, 0, budget_s)
    what = (f"the first {len(sample)} of {n_rep} replicas of the workload" if n_rep > 1 else "the workload")
    return {"value": va, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{ka} full collision intervals of {what} ({n} solvent) after 1 warm-up, {ea:.1f} s, "
                      f"FP64 C oracle on {cores} OpenMP threads",
            "seconds": ea, "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "single_thread": {"value": v1, "cores": 1, "intervals": k1, "seconds": e1}}


def run_reference(args, ws, rank):
    """The reference arm: the FP64 oracle on every host core (its OpenMP loops),
    each step one full collision interval of a bounded sample of the workload
    (a batch: its first replicas up to about 1 M solvent)."""
    if rank != 0:
        return
    from oracle import oracle
    oracle.build()
    sample, n, n_rep, desc = oracle_sample(args.workload, args.precision, max_particles=1_000_000)
    cores = oracle.set_threads(0)
    try:
        systems = [oracle_system(oracle, r, st) for r, st in sample]
        for _ in range(args.warmup):
            for o in systems:
                o.step(1)
        budget = 150.0
        times = []
        t_all = time.perf_counter()
        for k in range(args.steps):
            t0 = time.perf_counter()
            for o in systems:
                o.step(1)
            times.append(time.perf_counter() - t0)
            if time.perf_counter() - t_all > budget:
                break
    finally:
        oracle.set_threads(1)
    done = len(times)
    tot = sum(times)
    value = n * done / tot
    what = f"the first {len(sample)} of {n_rep} replicas ({n} solvent)" if n_rep > 1 else f"the workload ({n} solvent)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": done,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / done, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}", "n_solvent": n, "precision": "fp64 oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{done} of {args.steps} requested full intervals of {what} (time budget "
                                   f"{budget:.0f} s) after {args.warmup} warm-up, {cores} OpenMP threads",
                         "nproc": os.cpu_count(), "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


CELL_ORDER = "hilbert"


def make_system(api, reps, states, precision, stream):
    from paper_1608_04904_gb300 import network
    rigid = lambda b: None if b is not None and "network" in b else b
    s = api.System([dict(cfg=cfg, n=len(st[0]), colloids=col, bonds=bonds, body=rigid(body))
                    for (cfg, col, bonds, body), st in zip(reps, states)], precision=precision,
                   bucket_cap=reps[0][0].get("bucket_cap", 0), stream=stream)
    s.set_cell_order(CELL_ORDER)
    for r, (x, v, fl) in enumerate(states):
        s.set_state(r, x, v, fl)
    for r, (cfg, col, bonds, body) in enumerate(reps):
        if body is not None and "network" in body:
            net = body["network"]
            colors = network.color_links(net["links"], len(net["xb"]))
            s.set_network(r, net["xb"], net["vb"], net["mb"], net["eps_A"], net["eps_B"], net["catalytic"],
                          net["sigma"], net["links"], net["d"], colors)
    return s


def timed_run(api, torch, reps, states, precision, steps, warmup, flush, dev_index, sample_clocks,
              barrier, md_cluster=0, md_kernel=0):
    # a stream of its own: intervals replay as CUDA graphs (the legacy
    # default stream cannot be captured)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        return _timed_run(api, torch, reps, states, precision, steps, warmup, flush, dev_index, sample_clocks,
                          barrier, md_cluster, md_kernel, stream)


def _timed_run(api, torch, reps, states, precision, steps, warmup, flush, dev_index, sample_clocks,
               barrier, md_cluster, md_kernel, stream):
    s = make_system(api, reps, states, precision, stream)
    s.set_tuning(md_cluster, md_kernel)
    has_col = any(col for _, col, _, _ in reps)
    # warm-up, including the tuning intervals of the MD cluster size
    for _ in range(max(warmup, 16 if (has_col and md_cluster == 0) else 0)):   # 3 trials x <= 5 sizes
        s.step(1)
    torch.cuda.synchronize()
    # rigid bodies: centre of mass before the timed steps (for the MSD)
    body_reps = [r for r, rep in enumerate(reps) if rep[3] is not None]

    def com(r):
        body = reps[r][3]
        if "network" not in body:
            return s.get_body(r)["x"]
        xb, _ = s.get_network(r)
        m = body["network"]["mb"]
        return (m[:, None] * xb).sum(0) / m.sum()

    x0 = [com(r) for r in body_reps]
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    launches0 = s.launch_count()
    clk = ClockSampler(dev_index) if sample_clocks else None
    if clk:
        clk.start()
        time.sleep(0.25)
    barrier()
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        ev0[k].record(stream)
        s.step(1)
        ev1[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop() if clk else None
    launches = s.launch_count() - launches0
    msd = None
    if body_reps:
        import numpy as np
        d2 = np.array([float(((com(r) - a) ** 2).sum()) for r, a in zip(body_reps, x0)])
        msd = {"intervals": steps, "time": steps * reps[body_reps[0]][0]["tau"], "mean": float(d2.mean()),
               "min": float(d2.min()), "max": float(d2.max()), "replicas": len(d2),
               "per_replica_first8": [round(float(v), 6) for v in d2[:8]]}
    ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
    # per-kernel times: a further run with the library's timers (events
    # around each launch, so direct launches instead of graphs)
    s.enable_timers(True)
    s.read_timers(reset=True)
    for _ in range(min(steps, 200)):
        flush.zero_()
        s.step(1)
    timers = s.read_timers(reset=True)
    s.enable_timers(False)
    obs = s.observables(0)
    obs["md_cluster"], obs["md_kernel"] = s.get_tuning()
    obs["bucket_cap"] = s.bucket_cap()
    obs["msd"] = msd
    s.close()
    return ms, timers, launches, clocks, obs


def e2e_run(api, torch, reps, states, precision, steps):
    """Same metric through the public API with pinned host buffers: every step
    copies the whole state in (rmpcd_set_state_all), runs one interval and
    reads the whole state back (rmpcd_get_state_all)."""
    pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
    n = sum(len(st[0]) for st in states)
    bufs = []
    for _ in range(2):
        bufs.append({"x": pin((n, 3), torch.float64), "v": pin((n, 3), torch.float64),
                     "flags": pin((n,), torch.uint8)})
    off = 0
    for x, v, fl in states:
        k = len(x)
        bufs[0]["x"][off:off + k], bufs[0]["v"][off:off + k], bufs[0]["flags"][off:off + k] = x, v, fl
        off += k
    s = make_system(api, reps, states, precision, torch.cuda.current_stream())
    # one untimed round trip: the first interval and the staging area of the batch calls
    s.set_state_all(bufs[0]["x"], bufs[0]["v"], bufs[0]["flags"])
    s.step(1)
    s.get_state_all(out=bufs[1])
    bufs.reverse()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        hin, hout = bufs
        s.set_state_all(hin["x"], hin["v"], hin["flags"])
        s.step(1)
        s.get_state_all(out=hout)
        # the state read back is the next step's input
        bufs.reverse()
    el = time.perf_counter() - t0
    s.close()
    per = n * (24 + 24 + 1)
    return {"value": n * steps / el, "unit": UNIT, "h2d_bytes_per_step": per, "d2h_bytes_per_step": per,
            "steps": steps, "api": "rmpcd_set_state_all(host) + rmpcd_step(1) + rmpcd_get_state_all(host), pinned"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch256",
                    choices=["dimer32", "dimer64", "sphere16", "poiseuille128", "thermal", "batch256",
                             "network64"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--md-cluster", type=int, default=0, help="MD CTAs per replica (0 = autotune)")
    ap.add_argument("--md-kernel", type=int, default=0, help="MD kernel: 0 auto, 1 general, 2 few-colloid")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--bucket-cap", type=int, default=None,
                    help="cell row width (default: the automatic width)")
    ap.add_argument("--cell-order", default="hilbert", choices=["linear", "hilbert"],
                    help="storage order of the cells (rmpcd_set_cell_order; the paper sorts by compact "
                         "Hilbert index)")
    ap.add_argument("--replicas", type=int, default=None,
                    help="batch256 only: keep the first N replicas (a smaller case for profiling)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.workload == "network64":
        args.precision = "fp64"   # the network integrator is FP64 only
    global CELL_ORDER
    CELL_ORDER = args.cell_order
    ws, rank, local = dist_setup()

    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        barrier = lambda: dist.barrier()
    else:
        barrier = lambda: None

    from paper_1608_04904_gb300 import api, build, synth
    build.build()
    api.load()

    reps, desc = workload(args.workload, args.precision, seed_offset=rank, n_replicas=args.replicas)
    if args.bucket_cap is not None:
        for rep in reps:
            rep[0]["bucket_cap"] = args.bucket_cap
    states = [initial_state(r) for r in reps]
    cfg = reps[0][0]
    n = sum(len(st[0]) for st in states)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    ms, timers, launches, clocks, obs = timed_run(api, torch, reps, states, args.precision,
                                                  args.steps, args.warmup, flush, local, rank == 0, barrier,
                                                  args.md_cluster, args.md_kernel)
    value, ms_max = job_throughput(ms, n, args.steps, device="cuda")

    # roofline of the dominant kernel (CUDA events around each launch on the library's stream)
    phases = {k: v_ for k, v_ in timers.items() if v_["launches"] > 0}
    dominant = max(phases, key=lambda k: phases[k]["ms"])
    peak, peak_src = measured_peaks()
    kernel_names = dict(KERNEL_NAMES)
    if any(r[3] is not None and "network" in r[3] for r in reps):
        kernel_names["md"] = "k_md_network"
    elif any(r[3] is not None for r in reps):
        kernel_names["md"] = "k_md_body"
    elif obs["md_kernel"] == 2:
        kernel_names["md"] = "k_md_fast"
    kernels = {}
    for k, t in phases.items():
        avg_ms = t["ms"] / t["launches"]
        entry = {"launches": t["launches"], "avg_us": 1e3 * avg_ms, "share": t["ms"] / sum(p["ms"] for p in phases.values())}
        if k == "cellpass":
            alg = n * ALG_BYTES[args.precision]
            entry.update({"alg_bytes_per_launch": alg, "achieved_gbs": alg / (avg_ms / 1e3) / 1e9})
        if k == "md":
            entry["us_per_substep"] = 1e3 * avg_ms / max(r[0]["n_md"] for r in reps)
        kernels[kernel_names[k]] = entry
    cp = phases["cellpass"]
    cp_avg_s = cp["ms"] / cp["launches"] / 1e3
    alg = n * ALG_BYTES[args.precision]
    achieved = alg / cp_avg_s / 1e9
    roofline = {"kernel": "k_cellpass", "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": ncu_traffic("k_cellpass", args.workload, args.precision, n, args.cell_order),
                "peak_source": f"{peak_src} hbm_gbs", "dominant_kernel": kernel_names[dominant],
                "alg_bytes_per_particle": ALG_BYTES[args.precision]}
    if dominant == "md":
        md = phases["md"]
        roofline["note"] = ("%s (near-colloid velocity-Verlet: %d dependent sub-steps on one thread-block cluster, "
                            "%.2f us each) takes %.0f%% of the step and is latency-bound (no DRAM or ALU roof "
                            "applies); the HBM roofline reported is that of the cell pass, the bandwidth-bound "
                            "part of the step" % (kernel_names["md"], cfg["n_md"],
                                                  1e3 * md["ms"] / md["launches"] / cfg["n_md"],
                                                  100 * md["ms"] / sum(p["ms"] for p in phases.values())))

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}", "n_solvent": n, "n_replicas": len(reps),
                   "precision": args.precision,
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write, untimed)",
                   "timing": "CUDA events around each rmpcd_step(1) on the library's stream (intervals replayed "
                             "as CUDA graphs); per-kernel times from a further run with the library's timers",
                   "md_cluster": obs["md_cluster"], "md_kernel": obs["md_kernel"], "cell_order": args.cell_order,
                   "bucket_cap": obs["bucket_cap"]},
        "roofline": roofline, "kernels": kernels, "gpu_launches": launches, "clocks": clocks,
        "observables": {"temperature": obs["temperature"], "n_B": obs["n_B"], "kT": cfg["kT"]},
    }
    if obs.get("msd"):
        # mean squared displacement of the bodies' centres over the timed intervals (per replica)
        line["observables"]["body_msd"] = obs["msd"]
    if rank == 0 and not args.no_fp64 and args.precision == "mixed":
        k64 = max(20, args.steps // 4)
        ms64, t64, _, _, _ = timed_run(api, torch, reps, states, "fp64", k64, args.warmup, flush, local,
                                       False, lambda: None, args.md_cluster, args.md_kernel)
        v64 = n * k64 / (ms64 / 1e3)
        line["fp64"] = {"value": v64, "ms_per_step": ms64 / k64, "steps": k64,
                        "cellpass_avg_us": 1e3 * t64["cellpass"]["ms"] / t64["cellpass"]["launches"]}
        line["speedup_mixed_over_fp64"] = (n * args.steps / (ms / 1e3)) / v64
    if rank == 0 and not args.no_e2e:
        line["e2e"] = e2e_run(api, torch, reps, states, args.precision, min(args.steps, 200))
    if rank == 0 and not args.no_cpu and ws == 1:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.precision)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
