#!/usr/bin/env python
"""Throughput of the event-based Monte Carlo transport loop on GB300.

Workload: the C5G7-shaped 7-group lattice k-eigenvalue problem with synthetic
cross sections (2x2 assemblies of 17x17 pins plus reflector), 1e6 histories
per batch, 20 inactive + 50 active batches, 51x51x1 pin-mesh flux tally.  One
step is one complete power iteration of that workload (all batches: source,
lookup, distance, move, collide / cross, tally, remap, bank ordering,
splitting roulette).  The metric is particle events per second (collision and
surface outcomes; source events excluded) over the whole job.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank runs an independent replica with its own
seed (weak scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_PER_BATCH = 1_000_000
N_INACTIVE, N_ACTIVE = 20, 50
WORKLOAD = "c5g7-shaped 7-group lattice k-eigenvalue, 1e6 histories/batch, 20 inactive + 50 active batches"

# Algorithmic bytes per event of an event-based implementation: the particle
# record read and written once per event.  Multigroup: 64 B (position and
# direction 6 x 8 B; history index, event count, packed group and cell,
# problem index 4 x 4 B), so 2 x 64 = 128 B; the cross sections (3.5 KB) and
# the 20.8 KB tally stay on chip.  Continuous energy: a 72 B record (the
# energy added) both ways, plus the lookup's grid pair (16 B) and 16 B per
# (nuclide, reaction) term of the material (9 in the fuel): 304 B.
B_EVENT = {"lattice": 2 * 64, "ce": 2 * 72 + 16 + 16 * 9}

# The sources the measured kernels (k_presample and k_async, tr_async.cu and
# the headers it includes) are compiled from: the FP64-operation and
# DRAM-traffic figures below were measured on the sources with the digest
# stored beside them, and are reported as stale once the built sources differ.
TRANSPORT_SOURCES = ("tr_device.cuh", "tr_events.cuh", "tr_fixed.cuh", "tr_softfp.cuh", "tr_kernels.h", "tr_async.cu")


def kernel_digest(csrc=None):
    """SHA-256 (16 hex digits) over the transport kernels' source files."""
    import hashlib
    csrc = csrc or os.path.join(ROOT, "paper_2506_00263_gb300", "csrc")
    h = hashlib.sha256()
    for name in TRANSPORT_SOURCES:
        path = os.path.join(csrc, name)
        if os.path.exists(path):
            h.update(name.encode())
            with open(path, "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:16]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


# FP64 issue model of GB300 (measured: 2 FP64 add/mul/fma thread-operations per
# clock per SM; 152 SMs): peak = 152 * 2 * f_max.
FP64_OPS_PER_CLK_PER_SM = 2.0
N_SM = 152


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.samples.append([x.strip() for x in out.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        mhz = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for name, v in zip(names, s[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _cpu_baseline(seconds_budget: float = 15.0):
    """The oracle, as it stands, on a bounded sample of the same workload."""
    import oracle
    from paper_2506_00263_gb300 import inputs
    p = inputs.c5g7_lattice()
    nper, ni, na = 100_000, 4, 36       # about 10-20 s on one host core
    t0 = time.perf_counter()
    r = oracle.power_iteration(p, nper, ni, na, seed=1)
    dt = time.perf_counter() - t0
    ev = int(r["events_by_type"][1:].sum())
    out = {"value": ev / dt, "unit": "events/s", "cores": 1, "kind": "oracle",
           "sample": f"lattice power iteration, {nper} histories/batch x {ni + na} batches "
                     f"({ev} events, {dt:.1f} s, one host core)",
           "histories_per_s": nper * (ni + na) / dt}
    out["all_cores"] = _cpu_baseline_all_cores()
    return out


def _cpu_baseline_all_cores(n_total=1_600_000):
    """The same oracle on every host core: one batch's worth of lattice
    histories split into contiguous id ranges, one spawned process per core
    (the histories of a batch are independent); events/s over the slowest
    worker's time."""
    import multiprocessing as mp
    nproc = os.cpu_count() or 1
    per = max(n_total // nproc, 1)
    with mp.get_context("spawn").Pool(nproc) as pool:
        res = pool.map(_oracle_fixed_shard, [("lattice", per, i * per) for i in range(nproc)])
    ev = sum(e for e, _ in res)
    t = max(dt for _, dt in res)
    return {"value": ev / t, "unit": "events/s", "cores": nproc, "kind": "oracle",
            "sample": f"{per * nproc} lattice histories (fixed source, fission sites not iterated) over "
                      f"{nproc} contiguous id ranges, one spawned process per core ({ev} events, {t:.1f} s)"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_2506_00263_gb300 import inputs
    p = inputs.c5g7_lattice()
    nper, ni, na = 50_000, 1, 2          # a bounded sample of the workload per step
    for _ in range(args.warmup):
        oracle.power_iteration(p, nper, ni, na, seed=1)
    ev_tot, t_tot = 0, 0.0
    for k in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.power_iteration(p, nper, ni, na, seed=1 + k)
        t_tot += time.perf_counter() - t0
        ev_tot += int(r["events_by_type"][1:].sum())
    value = ev_tot / t_tot
    line = {"impl": "reference", "metric": "particle-events/s", "value": value, "unit": "events/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + f" (oracle sample: {nper}/batch x {ni + na} batches per step)",
                       "l2": "n/a (host)"},
            "cpu_baseline": {"value": value, "unit": "events/s", "cores": 1, "kind": "oracle",
                             "sample": f"{nper} histories/batch x {ni + na} batches per step, one core"},
            "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2506_00263_gb300 import binding as tb
    from paper_2506_00263_gb300 import build as tbuild
    from paper_2506_00263_gb300 import inputs

    if rank == 0 or not os.path.exists(tbuild.LIB):
        tbuild.build()
    if ws > 1:
        torch.distributed.barrier()
    scheme = tb.SCHEME_ASYNC if args.scheme == "async" else tb.SCHEME_STACK
    decomp = _DECOMPS[args.decomp]
    spec = inputs.c5g7_lattice()
    opts = tb.RunOpts(seed=1 + 1000 * rank, scheme=scheme, decomposition=decomp, stash_slots=args.stash,
                      blocks_per_sm=args.bps, remap_every=args.remap if args.decomp in ("mono", "stream") else 1,
                      queue_capacity=args.queue)
    stream = torch.cuda.current_stream()
    prob = tb.Problem(spec)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device="cuda")   # 512 MB > L2

    def step(p):
        return p.power_iteration(args.n_per_batch, args.inactive, args.active, opts)

    for _ in range(args.warmup):
        step(prob)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches0 = tb.kernel_launch_count()
    ev_tot = hist_tot = 0
    kern_s = 0.0
    kern_launches = 0
    times = []
    sampler = ClockSampler(torch.cuda.current_device())
    torch.cuda.synchronize()
    with sampler:
        for k in range(args.steps):
            flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = step(prob)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
            ev_tot += int(r["events"])
            hist_tot += int(r["histories"])
            kern_s += r["transport_seconds"]
            kern_launches += int(r["transport_launches"])
    torch.cuda.synchronize()
    launches = tb.kernel_launch_count() - launches0      # this library's kernels only (the L2 flush is torch's)
    t = sum(times)
    if ws > 1:
        from paper_2506_00263_gb300 import parallel
        t, ev_all, hist_all = parallel.reduce_timing(t, float(ev_tot), float(hist_tot), device="cuda")
    else:
        ev_all, hist_all = float(ev_tot), float(hist_tot)
    value = ev_all / t

    # ---- roofline of the dominant kernel (the transport loop, with the source
    # pre-sampling that feeds it: both run inside the timed launch bracket) ----
    hbm, fmax, peak_kind = _peaks()
    avg_launch = kern_s / max(kern_launches, 1)
    ev_per_launch = ev_tot / max(kern_launches, 1)
    bench_cfg = (args.scheme, args.decomp, opts.remap_every, args.n_per_batch) == ("async", "mono", 512, N_PER_BATCH)
    traffic, traffic_fresh = measured_figure(TRAFFIC, "lattice")
    traffic = traffic if (traffic_fresh and bench_cfg) else None
    hbm_roof = _hbm_roof(ev_per_launch, avg_launch, "lattice", traffic)
    alu_roof = _alu_roof("lattice", ev_per_launch, avg_launch,
                         "FP64 pipe (add/mul/fma) of one batch's transport (source pre-sampling + transport loop)",
                         traffic)
    # the binding roof is the FP64 pipe; its per-event operation count is an
    # ncu measurement and counts only while it describes the built kernels
    roof = alu_roof if (alu_roof and not alu_roof.get("stale")) else hbm_roof

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if rank == 0 and args.e2e_steps > 0:
        pinned_spec, h2d = _pinned_copy(spec, torch)
        torch.cuda.synchronize()
        ev_e, t_e = 0, 0.0
        d2h = 0
        for k in range(args.e2e_steps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p2 = tb.Problem(pinned_spec)
            r = step(p2)
            mesh = p2.tally(tb.TALLY_MESH)
            sc = p2.tally(tb.TALLY_SCALARS)
            p2.close()
            torch.cuda.synchronize()
            t_e += time.perf_counter() - t0
            ev_e += int(r["events"])
            d2h = mesh.nbytes + sc.nbytes + 3 * 8 * (args.inactive + args.active)
        e2e = {"value": ev_e / t_e, "unit": "events/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---- the other reported quantities (not part of the timed value) ----
    # (the benchmark problem is released first: with it alive, the CE pin
    # cell's transport measured 16 % slower)
    prob.close()
    extras = None
    if rank == 0 and not args.no_extras:
        ce = measure_ce_line(torch, tb, inputs)
        paper = measure_paper_setting(torch, tb, spec)
        adj = measure_adjoint(torch, tb, inputs, 3, 2, decomp)
        bat = measure_batched(torch, tb, inputs, 2, 2, decomp)
        extras = {
            "paper_setting": paper,
            "ce_pin_cell": ce,
            "gradient": {"workload": ADJ_WORKLOAD, "forward_ms": adj["forward_ms"], "backward_ms": adj["backward_ms"],
                         "gradient_over_forward": adj["gradient_over_forward"]},
            "batched": {"workload": BATCH_WORKLOAD, "events_per_s": bat["events_per_s"],
                        "ms_per_call": 1e3 * bat["seconds"] / 2, "first_call_s": bat["first_call_s"],
                        "tuning_used": bat["tuning_used"],
                        "sequential_single_runs_events_per_s": bat["sequential_single_runs"]["events_per_s"],
                        "speedup_of_batched": bat["sequential_single_runs"]["speedup_of_batched"]}}
    if rank != 0:
        return 0
    cpu = None if args.no_cpu_baseline else _cpu_baseline()
    line = {
        "metric": "particle-events/s", "value": value, "unit": "events/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "scheme": args.scheme, "decomposition": args.decomp,
                   "stash_slots": args.stash, "blocks_per_sm": args.bps,
                   "remap_every": args.remap if args.decomp in ("mono", "stream") else 1,
                   "n_per_batch": args.n_per_batch, "batches": args.inactive + args.active,
                   "l2": "flushed between steps (512 MB write)"},
        "histories_per_s": hist_all / t,
        "roofline": roof, "hbm_roofline": hbm_roof, "alu_roofline": alu_roof,
        "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": launches,
        "clocks": sampler.summary(),
        "transport": {"kernel_seconds": kern_s, "launches": kern_launches, "avg_launch_ms": 1e3 * avg_launch},
        "extras": extras,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


PAPER_BATCHES = (2, 6)   # inactive, active batches of the paper-setting comparison (1e6 histories each)


def measure_paper_setting(torch, tb, spec, n_per_batch=N_PER_BATCH):
    """The lattice power iteration at the paper's setting, one event per remap
    (whole events per pass), with asynchronous and stack-based remapping, and
    with the default 512 events per remap, on the same batches: events/s of
    each (CUDA events around the whole power iteration)."""
    stream = torch.cuda.current_stream()
    prob = tb.Problem(spec)
    out = {"workload": f"the benchmark lattice, {n_per_batch} histories/batch, {PAPER_BATCHES[0]} inactive + "
                       f"{PAPER_BATCHES[1]} active batches"}
    for label, scheme, remap in (("async_1_event_per_remap", tb.SCHEME_ASYNC, 1),
                                 ("stack_1_event_per_remap", tb.SCHEME_STACK, 1),
                                 ("async_512_events_per_remap", tb.SCHEME_ASYNC, 512)):
        opts = tb.RunOpts(seed=1, scheme=scheme, decomposition=tb.DECOMP_MONO, remap_every=remap)
        prob.power_iteration(n_per_batch, 1, 2, opts)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = prob.power_iteration(n_per_batch, PAPER_BATCHES[0], PAPER_BATCHES[1], opts)
        e1.record(stream)
        e1.synchronize()
        out[label] = int(r["events"]) / (e0.elapsed_time(e1) * 1e-3)
    prob.close()
    out["async_over_stack_at_1_event_per_remap"] = out["async_1_event_per_remap"] / out["stack_1_event_per_remap"]
    return out


def measure_ce_line(torch, tb, inputs, n=1_000_000, steps=3):
    """The continuous-energy pin cell (1e6 histories, 100 energy bins,
    asynchronous monolithic, 64 events per remap): events/s and rooflines."""
    prob = tb.Problem(inputs.ce_pin_cell(n_ebins=100))
    opts = tb.RunOpts(n_histories=n, seed=1, scheme=tb.SCHEME_ASYNC, decomposition=tb.DECOMP_MONO, remap_every=64)
    with ClockSampler(torch.cuda.current_device()) as sampler:
        t, ev = _time_fixed(torch, tb, prob, opts, steps, 2)
    prob.close()
    return {"workload": CE_WORKLOAD + f", {n} histories, 100 bins, 64 events per remap",
            "events_per_s": ev / t, "histories_per_s": n * steps / t, "clocks": sampler.summary(),
            "hbm_roofline": _hbm_roof(ev / steps, t / steps, "ce", _fresh_traffic("ce")),
            "alu_roofline": _alu_roof("ce", ev / steps, t / steps, "FP64 pipe (add/mul/fma) of the run",
                                      _fresh_traffic("ce"))}


BATCH_WORKLOAD = ("256 independent multigroup voxel boxes (groups from {1,2,7,20,70}, 1-8 materials, "
                  "up to 64^3 voxels, 1e3-1e6 histories log-uniform, 8^3-32^3 mesh) in one batched launch")
ADJ_WORKLOAD = ("differentiated 7-group lattice, fission off, uniform source in fuel pins, 1e6 histories: "
                "forward fixed-source run + derivatives of the 51x51 mesh flux and absorption rate")


def _setup(torch):
    """Process group (N > 1), device, library build; returns (ws, rank, tb, inputs)."""
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2506_00263_gb300 import binding as tb
    from paper_2506_00263_gb300 import build as tbuild
    from paper_2506_00263_gb300 import inputs
    if rank == 0 or not os.path.exists(tbuild.LIB):
        tbuild.build()
    if ws > 1:
        torch.distributed.barrier()
    return ws, rank, tb, inputs


def measure_batched(torch, tb, inputs, steps, warmup, decomp, seed=1, tuning=(0, 0, 0), sampler=None,
                    barrier=None):
    """One step = one tr_run_batched over the 256-problem workload (autotuned
    and graph-replayed after the first call), timed with CUDA events; then
    the same problems once more, one tr_run_fixed_source after another."""
    specs, hist = inputs.batched_boxes(256, seed=7 + seed)
    probs = [tb.Problem(s) for s in specs]
    bps, stash, remap = tuning
    opts = tb.RunOpts(seed=seed, scheme=tb.SCHEME_ASYNC, decomposition=decomp, stash_slots=stash,
                      blocks_per_sm=bps, remap_every=remap)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device="cuda")
    t_first = time.perf_counter()
    tb.run_batched(probs, hist, opts)            # autotuning + graph capture
    t_first = time.perf_counter() - t_first
    for _ in range(warmup):
        tb.run_batched(probs, hist, opts)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    launches0 = tb.kernel_launch_count()
    times, ev_tot, kern_s = [], 0, 0.0
    import contextlib
    with (sampler or contextlib.nullcontext()):
        for k in range(steps):
            flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = tb.run_batched(probs, hist, opts)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
            ev_tot += sum(int(s["events"]) for s in st)
            kern_s += st[0]["transport_seconds"]
    torch.cuda.synchronize()
    launches = tb.kernel_launch_count() - launches0
    used = st[0]["used"]
    single = lambda n, i: tb.RunOpts(n_histories=n, seed=seed, scheme=tb.SCHEME_ASYNC, decomposition=decomp,
                                     problem_tag=i)
    for i, (p, n) in enumerate(zip(probs, hist)):      # warm
        p.run_fixed_source(single(min(n, 1000), i))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ev_seq = 0
    for i, (p, n) in enumerate(zip(probs, hist)):
        ev_seq += int(p.run_fixed_source(single(n, i))["events"])
    e1.record(stream)
    e1.synchronize()
    t_seq = e0.elapsed_time(e1) * 1e-3
    for p in probs:
        p.close()
    t = sum(times)
    return {"seconds": t, "events": ev_tot, "histories": float(sum(hist)) * steps, "kernel_seconds": kern_s,
            "launches": launches, "first_call_s": t_first, "problems": len(specs),
            "tuning_used": {"blocks_per_sm": used[0], "stash_slots": used[1], "remap_every": used[2]},
            "events_per_s": ev_tot / t,
            "sequential_single_runs": {"events_per_s": ev_seq / t_seq, "seconds": t_seq,
                                       "speedup_of_batched": (ev_tot / t) / (ev_seq / t_seq)}}


def measure_adjoint(torch, tb, inputs, steps, warmup, decomp, seed=1, sampler=None, barrier=None):
    """One step = one forward and one backward pass through TransportFn
    (torch.autograd) on the fission-off lattice, 1e6 histories: the forward
    pass writes the cross sections (CUDA tensors) into a kept problem on the
    device and runs the fixed-source transport; the backward pass of
    L = g . mesh + absorption rate runs the derivative kernels.  Forward and
    backward are timed separately with CUDA events on the stream."""
    import contextlib
    import numpy as np
    from paper_2506_00263_gb300.autograd import transport
    spec = inputs.c5g7_lattice(fission=False)
    opts = tb.RunOpts(n_histories=1_000_000, seed=seed, scheme=tb.SCHEME_ASYNC, decomposition=decomp,
                      remap_every=512 if decomp == tb.DECOMP_MONO else 1)
    prob = tb.Problem(spec)
    xs0 = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in (spec.sigma_t, spec.sigma_s,
                                                                           spec.nu_sigma_f)]
    g_mesh = torch.tensor(np.random.default_rng(3).uniform(-1, 1, spec.mesh_size), dtype=torch.float64,
                          device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device="cuda")

    def one_step(events=None):
        xs = [x.clone().requires_grad_(True) for x in xs0]
        if events:
            events[0].record(stream)
        mesh, scal = transport(xs[0], xs[1], xs[2], prob, opts)
        if events:
            events[1].record(stream)
        ((mesh * g_mesh).sum() + scal[1]).backward()
        if events:
            events[2].record(stream)
        return xs

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize()
    if barrier:
        barrier()
    launches0 = tb.kernel_launch_count()
    t_f = t_b = 0.0
    ev = 0
    with (sampler or contextlib.nullcontext()):
        for k in range(steps):
            flush.fill_(float(k))
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            one_step(e)
            e[2].synchronize()
            t_f += e[0].elapsed_time(e[1]) * 1e-3
            t_b += e[1].elapsed_time(e[2]) * 1e-3
            ev += int(prob.last_stats["events"])
    launches = tb.kernel_launch_count() - launches0
    prob.close()
    return {"seconds": t_f + t_b, "events": ev, "launches": launches, "forward_ms": 1e3 * t_f / steps,
            "backward_ms": 1e3 * t_b / steps, "gradient_over_forward": t_b / t_f,
            "forward_events_per_s": ev / t_f, "through": "torch.autograd (TransportFn forward + backward)"}


def _side_line(args, ws, workload, m, t, ev_all, hist_all, sampler, roof, extra):
    return {"metric": "particle-events/s", "value": ev_all / t, "unit": "events/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict({"workload": workload, "decomposition": args.decomp,
                            "l2": "flushed between steps (512 MB write)"}, **extra),
            "histories_per_s": hist_all / t if hist_all else None, "roofline": roof, "e2e": None,
            "cpu_baseline": None, "gpu_launches": m["launches"], "clocks": sampler.summary()}


def _hbm_roof(ev, seconds, workload="lattice", traffic=None):
    """HBM roofline: algorithmic bytes per event (B_EVENT) times events over
    the device time, against the measured copy bandwidth."""
    hbm, _, peak_kind = _peaks()
    b = B_EVENT[workload]
    ach = b * ev / seconds / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": traffic,
            "target_frac": 0.5,
            "what": f"{b} algorithmic bytes/event (particle record read and written once), {peak_kind} peak"}


def _alu_roof(workload, ev, seconds, what, traffic=None):
    """FP64-pipe roofline: executed FP64 operations per event (an ncu
    measurement of the kernels with the recorded source digest) times events
    over the device time, against 152 SMs x 2 FP64 operations per clock at the
    maximum SM clock.  Marked stale when the kernels changed since."""
    ops, fresh = measured_figure(FP64_OPS, workload)
    if ops is None:
        return None
    _, fmax, _ = _peaks()
    peak = N_SM * FP64_OPS_PER_CLK_PER_SM * fmax * 1e6 / 1e12
    ach = ops * ev / seconds / 1e12
    r = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": traffic,
         "what": f"{what}, {ops:g} FP64 ops/event (ncu, kernels {FP64_OPS[workload][1]})",
         "peak_source": f"derived: {N_SM} SMs x {FP64_OPS_PER_CLK_PER_SM:g} FP64/clk x {fmax:.0f} MHz"}
    if not fresh:
        r["stale"] = f"measured on kernels {FP64_OPS[workload][1]}, built kernels are {kernel_digest()}"
    return r


def run_batched_workload(args):
    import torch
    ws, rank, tb, inputs = _setup(torch)
    decomp = tb.DECOMP_SPLIT if args.decomp == "split" else tb.DECOMP_MONO
    sampler = ClockSampler(torch.cuda.current_device())
    m = measure_batched(torch, tb, inputs, args.steps, args.warmup, decomp, seed=1 + 1000 * rank,
                        tuning=(args.bps, args.stash, args.remap if args.bps else 0), sampler=sampler,
                        barrier=torch.distributed.barrier if ws > 1 else None)
    t, ev_all, hist_all = m["seconds"], float(m["events"]), m["histories"]
    if ws > 1:
        from paper_2506_00263_gb300 import parallel
        t, ev_all, hist_all = parallel.reduce_timing(t, ev_all, hist_all, device="cuda")
    if rank == 0:
        line = _side_line(args, ws, BATCH_WORKLOAD, m, t, ev_all, hist_all, sampler,
                          _hbm_roof(m["events"], m["kernel_seconds"], "lattice"),
                          {"problems": m["problems"], "tuning_used": m["tuning_used"]})
        line.update({"first_call_s": m["first_call_s"], "sequential_single_runs": m["sequential_single_runs"],
                     "transport": {"kernel_seconds": m["kernel_seconds"], "launches": args.steps}})
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_adjoint_workload(args):
    import torch
    ws, rank, tb, inputs = _setup(torch)
    decomp = _DECOMPS[args.decomp]
    sampler = ClockSampler(torch.cuda.current_device())
    m = measure_adjoint(torch, tb, inputs, args.steps, args.warmup, decomp, seed=1 + 1000 * rank, sampler=sampler,
                        barrier=torch.distributed.barrier if ws > 1 else None)
    t, ev_all = m["seconds"], float(m["events"])
    if ws > 1:
        from paper_2506_00263_gb300 import parallel
        t, ev_all, _ = parallel.reduce_timing(t, ev_all, 0.0, device="cuda")
    if rank == 0:
        line = _side_line(args, ws, ADJ_WORKLOAD, m, t, ev_all, None, sampler,
                          _hbm_roof(m["events"], m["forward_ms"] * 1e-3 * args.steps, "lattice"), {})
        line.update({k: m[k] for k in ("forward_ms", "backward_ms", "gradient_over_forward")})
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


CE_WORKLOAD = ("continuous-energy infinite pin cell (4 synthetic nuclides, 1e5 points and 300 resonances each, "
               "union grid ~4e5), Watt-like source in the fuel, energy tally per material")
_DECOMPS = {"mono": 0, "split": 1, "lookup": 2, "stream": 3}


def _time_fixed(torch, tb, prob, opts, steps, warmup):
    """Device time (CUDA events) of `steps` fixed-source runs after `warmup`."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        prob.run_fixed_source(opts)
    torch.cuda.synchronize()
    t, ev = 0.0, 0
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = prob.run_fixed_source(opts)
        e1.record(stream)
        e1.synchronize()
        t += e0.elapsed_time(e1) * 1e-3
        ev += int(r["events"])
    return t, ev


def run_ce_workload(args):
    """One step = one fixed-source run of the CE pin cell (args.n_hist histories,
    args.ebins energy bins) with the chosen scheme and decomposition."""
    import torch
    ws, rank, tb, inputs = _setup(torch)
    spec = inputs.ce_pin_cell(n_ebins=args.ebins)
    prob = tb.Problem(spec)
    opts = tb.RunOpts(n_histories=args.n_hist, seed=1 + 1000 * rank,
                      scheme=tb.SCHEME_ASYNC if args.scheme == "async" else tb.SCHEME_STACK,
                      decomposition=_DECOMPS[args.decomp], remap_every=args.remap if args.decomp in ("mono", "stream") else 1)
    sampler = ClockSampler(torch.cuda.current_device())
    launches0 = tb.kernel_launch_count()
    with sampler:
        t, ev = _time_fixed(torch, tb, prob, opts, args.steps, args.warmup)
    m = {"launches": tb.kernel_launch_count() - launches0}
    ev_all = float(ev)
    if ws > 1:
        from paper_2506_00263_gb300 import parallel
        t, ev_all, _ = parallel.reduce_timing(t, ev_all, 0.0, device="cuda")
    if rank == 0:
        measured_cfg = (args.scheme, args.decomp, args.ebins, opts.remap_every, args.n_hist) == \
            ("async", "mono", 100, 64, 1_000_000)
        traffic = _fresh_traffic("ce") if measured_cfg else None
        roof = _hbm_roof(ev / args.steps, t / args.steps, "ce", traffic)
        if measured_cfg:
            alu = _alu_roof("ce", ev / args.steps, t / args.steps,
                            "FP64 pipe (add/mul/fma) of the run (asynchronous monolithic, 100 bins)", traffic)
            roof = alu if (alu and not alu.get("stale")) else roof
        line = _side_line(args, ws, CE_WORKLOAD, m, t, ev_all, float(args.n_hist) * args.steps * ws, sampler, roof,
                          {"scheme": args.scheme, "energy_bins": args.ebins,
                           "histories": args.n_hist, "remap_every": opts.remap_every})
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_ce_sweep(args):
    """The paper's continuous-energy comparison (Sec. 5.2) on the synthetic pin
    cell: events/s for stack and asynchronous remapping under the monolithic,
    decomposed and lookup-event decompositions, over histories x energy-bin
    resolution, with each point's speedup over stack remapping with the
    monolithic scheme.  One JSON line per point."""
    import torch
    ws, rank, tb, inputs = _setup(torch)
    if rank != 0:
        return 0
    for nb in (1, 100, 10000):
        prob = tb.Problem(inputs.ce_pin_cell(n_ebins=nb))
        for n in (100_000, 1_000_000, 10_000_000):
            base = None
            for scheme in ("stack", "async"):
                for dname in ("mono", "split", "lookup"):
                    opts = tb.RunOpts(n_histories=n, seed=1, decomposition=_DECOMPS[dname], remap_every=1,
                                      scheme=tb.SCHEME_ASYNC if scheme == "async" else tb.SCHEME_STACK)
                    t, ev = _time_fixed(torch, tb, prob, opts, 1 if n >= 10_000_000 else 2, 1)
                    rate = ev / t
                    if base is None:
                        base = rate
                    print(json.dumps({"workload": "ce-sweep", "energy_bins": nb, "histories": n, "scheme": scheme,
                                      "decomposition": dname, "events_per_s": rate,
                                      "speedup_vs_stack_mono": rate / base}), flush=True)
        prob.close()
    return 0


def run_ce_time_sweep(args):
    """The paper's temporal tally resolution (Sec. 4): the CE pin cell with a
    14 MeV source and a census at 1 microsecond, over time-tally widths 1..128
    (powers of two) and histories, for stack and asynchronous remapping under
    the three decompositions, with each point's speedup over stack remapping
    with the monolithic scheme.  One JSON line per point."""
    import torch
    ws, rank, tb, inputs = _setup(torch)
    if rank != 0:
        return 0
    base_spec = inputs.ce_pin_cell(n_ebins=1, source_energy=14e6)
    for nb in (1, 2, 4, 8, 16, 32, 64, 128):
        prob = tb.Problem(base_spec.replace(t_census=1e-6, n_time_bins=nb))
        for n in (100_000, 1_000_000):
            base = None
            for scheme in ("stack", "async"):
                for dname in ("mono", "split", "lookup"):
                    opts = tb.RunOpts(n_histories=n, seed=1, decomposition=_DECOMPS[dname], remap_every=1,
                                      scheme=tb.SCHEME_ASYNC if scheme == "async" else tb.SCHEME_STACK)
                    t, ev = _time_fixed(torch, tb, prob, opts, 2, 1)
                    rate = ev / t
                    if base is None:
                        base = rate
                    print(json.dumps({"workload": "ce-time-sweep", "time_bins": nb, "histories": n,
                                      "scheme": scheme, "decomposition": dname, "events_per_s": rate,
                                      "speedup_vs_stack_mono": rate / base}), flush=True)
        prob.close()
    return 0


def _oracle_fixed_shard(args):
    """Worker of the all-core oracle timing (spawned process): one id range."""
    name, n, offset = args
    import oracle
    from paper_2506_00263_gb300 import inputs
    spec = {"cube": inputs.cube_one_group, "lattice": lambda: inputs.c5g7_lattice(fission=False),
            "ce": lambda: inputs.ce_pin_cell()}[name]()
    t0 = time.perf_counter()
    r = oracle.run_fixed_source(spec, n, seed=1, id_offset=offset, logs=False)
    return int(r["events_by_type"][1:].sum()), time.perf_counter() - t0


def run_baseline_table(args):
    """Per configuration: GPU events/s and histories/s (CUDA events, default
    tuning), FP64-issue and HBM roofline fractions, and the oracle's events/s
    on one host core and on all host cores (a spawned process pool over
    contiguous id ranges; fixed-source histories, the lattice without fission
    standing in for its eigenvalue batches).  One JSON line per row."""
    import multiprocessing as mp
    nproc = os.cpu_count() or 1
    pool = mp.get_context("spawn").Pool(nproc)      # started before any GPU work
    import oracle
    oracle.lib()                                      # built once, before the workers load it
    import torch
    ws, rank, tb, inputs = _setup(torch)
    if rank != 0:
        return 0
    hbm, fmax, _ = _peaks()
    fp64_peak = N_SM * FP64_OPS_PER_CLK_PER_SM * fmax * 1e6

    def oracle_rates(name, n1, nall):
        ev1, t1 = _oracle_fixed_shard((name, n1, 0))
        per = max(nall // nproc, 1)
        res = pool.map(_oracle_fixed_shard, [(name, per, i * per) for i in range(nproc)])
        return ev1 / t1, sum(e for e, _ in res) / max(t for _, t in res)

    rows = []
    # C1 cube, C3 CE pin cell (fixed source)
    for label, name, spec, n, remap in (("C1 one-group cube", "cube", inputs.cube_one_group(), 100_000, 512),
                                        ("C3 CE pin cell", "ce", inputs.ce_pin_cell(), 1_000_000, 64)):
        prob = tb.Problem(spec)
        opts = tb.RunOpts(n_histories=n, seed=1, scheme=tb.SCHEME_ASYNC, decomposition=tb.DECOMP_MONO,
                          remap_every=remap)
        t, ev = _time_fixed(torch, tb, prob, opts, 3, 2)
        prob.close()
        o1, oall = oracle_rates(name, 20_000 if name == "cube" else 2_000, 200_000 if name == "cube" else 20_000)
        rows.append({"config": label, "gpu_events_per_s": ev / t, "gpu_histories_per_s": 3 * n / t,
                     "oracle_1core_events_per_s": o1, "oracle_allcore_events_per_s": oall, "cores": nproc})
    # C2 lattice power iteration, both schemes
    prob = tb.Problem(inputs.c5g7_lattice())
    stream = torch.cuda.current_stream()
    for scheme in ("async", "stack"):
        opts = tb.RunOpts(seed=1, scheme=tb.SCHEME_ASYNC if scheme == "async" else tb.SCHEME_STACK,
                          decomposition=tb.DECOMP_MONO, remap_every=512 if scheme == "async" else 3)
        prob.power_iteration(1_000_000, 2, 2, opts)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = prob.power_iteration(1_000_000, 5, 10, opts)
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        rows.append({"config": f"C2 7-group lattice, {scheme}", "gpu_events_per_s": r["events"] / t,
                     "gpu_histories_per_s": r["histories"] / t})
    prob.close()
    o1, oall = oracle_rates("lattice", 10_000, 100_000)
    rows[-2].update({"oracle_1core_events_per_s": o1, "oracle_allcore_events_per_s": oall, "cores": nproc})
    # C4 batched, C5 gradient
    bat = measure_batched(torch, tb, inputs, 2, 2, tb.DECOMP_MONO)
    rows.append({"config": "C4 batched 256 boxes", "gpu_events_per_s": bat["events_per_s"],
                 "gpu_histories_per_s": bat["histories"] / bat["seconds"],
                 "vs_one_by_one": bat["sequential_single_runs"]["speedup_of_batched"]})
    adj = measure_adjoint(torch, tb, inputs, 3, 2, tb.DECOMP_MONO)
    rows.append({"config": "C5 gradient / forward time", "gradient_over_forward": adj["gradient_over_forward"],
                 "forward_ms": adj["forward_ms"], "backward_ms": adj["backward_ms"]})
    # FP64 fraction where the operation count was measured for the configuration
    kinds = {"C2 7-group lattice, async": "lattice", "C2 7-group lattice, stack": "lattice", "C3 CE pin cell": "ce",
             "C1 one-group cube": "lattice"}
    for r in rows:
        kind = kinds.get(r["config"])
        if kind:
            r["hbm_fraction"] = r["gpu_events_per_s"] * B_EVENT[kind] / (hbm * 1e9)
            ops, fresh = measured_figure(FP64_OPS, kind)
            if ops and r["config"] != "C1 one-group cube":
                r["fp64_issue_fraction"] = r["gpu_events_per_s"] * ops / fp64_peak
                if not fresh:
                    r["fp64_issue_fraction_stale"] = True
        print(json.dumps(r), flush=True)
    pool.close()
    return 0


def run_lattice_sweep(args):
    """The paper's multigroup comparison (Sec. 5.1): power iterations of the
    lattice with 25 % inactive cycles, over particles per cycle and cycle
    counts, asynchronous vs stack remapping (monolithic scheme, one event per
    remap as in the paper); one JSON line per point."""
    import torch
    ws, rank, tb, inputs = _setup(torch)
    if rank != 0:
        return 0
    prob = tb.Problem(inputs.c5g7_lattice())
    stream = torch.cuda.current_stream()
    for cycles in (24, 48, 100, 200, 400):
        ni = cycles // 4
        for nper in (10_000, 100_000, 1_000_000):
            if nper * cycles > 100_000_000:
                continue
            rates = {}
            for scheme in ("stack", "async"):
                opts = tb.RunOpts(seed=1, scheme=tb.SCHEME_ASYNC if scheme == "async" else tb.SCHEME_STACK,
                                  decomposition=tb.DECOMP_MONO, remap_every=1)
                prob.power_iteration(nper, 1, 2, opts)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = prob.power_iteration(nper, ni, cycles - ni, opts)
                e1.record(stream)
                e1.synchronize()
                rates[scheme] = int(r["events"]) / (e0.elapsed_time(e1) * 1e-3)
            print(json.dumps({"workload": "lattice-sweep", "cycles": cycles, "particles_per_cycle": nper,
                              "stack_events_per_s": rates["stack"], "async_events_per_s": rates["async"],
                              "async_speedup": rates["async"] / rates["stack"]}), flush=True)
    prob.close()
    return 0


# FP64 thread-operations (dadd + dmul + dfma, divisions and square roots
# included as executed) per transport event, from an ncu capture
# (sm__sass_thread_inst_executed_ops_dadd_dmul_dfma_pred_on.sum / events) of
# the source pre-sampling and transport kernels: the lattice power iteration
# (asynchronous monolithic, 512 events between remaps) and the CE pin cell
# (1e6 histories, 100 bins, 64 events between remaps).  Each figure carries
# the kernel_digest() of the sources it was measured on.
FP64_OPS = {"lattice": (52.1, "2b3524419633bdfe"), "ce": (94.1, "2b3524419633bdfe")}
# DRAM bytes (read + write), dram__bytes_read.sum + dram__bytes_write.sum, of
# one 1e6-history lattice batch's transport (source pre-sampling and transport
# kernels, asynchronous monolithic, 512 events between remaps; the mean of the
# timed step's three batches) and of one 1e6-history CE pin-cell run (the same
# two kernels, 64 events between remaps, 100 energy bins).
TRAFFIC = {"lattice": (248.5e6, "2b3524419633bdfe"), "ce": (223.2e6, "2b3524419633bdfe")}


def _fresh_traffic(key):
    """The measured DRAM bytes per launch of `key`, or None once the kernels changed."""
    v, fresh = measured_figure(TRAFFIC, key)
    return v if fresh else None


def measured_figure(table, key):
    """(value, fresh) of a measured per-kernel figure: fresh when it was
    measured on the sources built now."""
    if key not in table:
        return None, False
    value, digest = table[key]
    return value, digest == kernel_digest()


def _pinned_copy(spec, torch):
    """The problem's arrays copied into page-locked host memory; returns the
    spec and the bytes the library uploads."""
    import numpy as np
    nbytes = 0
    kw = {}
    for name in ("x_planes", "y_planes", "z_planes", "cell_material", "pin_material", "sigma_t", "sigma_s",
                 "nu_sigma_f", "chi", "src_materials"):
        a = getattr(spec, name)
        if a is None:
            continue
        t = torch.empty(a.shape, dtype={np.dtype("float64"): torch.float64, np.dtype("int32"): torch.int32,
                                        np.dtype("uint8"): torch.uint8}[a.dtype], pin_memory=True)
        t.numpy()[...] = a
        kw[name] = t.numpy()
        nbytes += a.nbytes
    return spec.replace(**kw), nbytes


ISSUE_OPS = {0: "dadd", 1: "dmul", 2: "dfma", 3: "ddiv", 4: "dsqrt", 5: "ffma", 6: "imad",
             8: "drcp (IEEE sequence)", 9: "drcp (sf_rcp, integer pipe)", 10: "dsqrt (IEEE sequence)",
             11: "dsqrt (sf_sqrt, integer pipe)"}


def run_issue_rate(args):
    """The arithmetic pipes' issue rates (the roofline's ALU denominators):
    one JSON line per operation, then the FP64 fma issued by 1..32 lanes of a
    warp (warp instructions per second), with the SM clock sampled during it."""
    import torch
    _, _, tb, _ = _setup(torch)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    reps = max(args.steps, 3)          # best of `reps` timed launches per operation
    with ClockSampler(0) as sampler:
        rows = [{"op": name, "per_s": max(tb.issue_rate(op) for _ in range(reps))}
                for op, name in ISSUE_OPS.items()]
        lanes = [{"lanes": k, "warp_instr_per_s": max(tb.issue_rate(7, k) for _ in range(reps))}
                 for k in (1, 2, 4, 8, 16, 32)]
    clocks = sampler.summary()
    mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz")
    for r in rows:
        r["per_clk_per_sm"] = r["per_s"] / (sms * mhz * 1e6) if mhz else None
        print(json.dumps(dict({"workload": "issue-rate"}, **r)))
    print(json.dumps({"workload": "issue-rate", "partial_warp_dfma": lanes, "sms": sms, "clocks": clocks}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scheme", choices=["async", "stack"], default="async")
    ap.add_argument("--decomp", choices=["split", "mono", "lookup", "stream"], default="mono")
    ap.add_argument("--n-per-batch", type=int, default=N_PER_BATCH)
    ap.add_argument("--inactive", type=int, default=N_INACTIVE)
    ap.add_argument("--active", type=int, default=N_ACTIVE)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the gradient and batched side measurements")
    ap.add_argument("--stash", type=int, default=0, help="async: particle slots per block stash (0 = default)")
    ap.add_argument("--bps", type=int, default=0, help="blocks per SM (0 = default)")
    ap.add_argument("--remap", type=int, default=0,
                    help="monolithic / streaming: events between remaps (0: 512 for the lattice, 64 for the CE pin cell)")
    ap.add_argument("--queue", type=int, default=0, help="stack: particles per stack; async: spill links x 32")
    ap.add_argument("--workload", choices=["lattice", "batched", "adjoint", "ce", "ce-sweep", "ce-time-sweep",
                                           "lattice-sweep", "baseline-table", "issue-rate"],
                    default="lattice",
                    help="lattice: the k-eigenvalue lattice; batched: 256 box problems in one launch; "
                         "adjoint: forward + derivative kernels on the fixed-source lattice; ce: the continuous-"
                         "energy pin cell; ce-sweep / lattice-sweep: the paper's scheme comparisons")
    ap.add_argument("--ebins", type=int, default=100, help="ce: energy-tally bins per material")
    ap.add_argument("--n-hist", type=int, default=1_000_000, help="ce: histories per run")
    args = ap.parse_args()
    if args.remap <= 0:
        args.remap = 64 if args.workload.startswith("ce") else 512
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched_workload(args)
    if args.workload == "adjoint":
        return run_adjoint_workload(args)
    if args.workload == "ce":
        return run_ce_workload(args)
    if args.workload == "ce-sweep":
        return run_ce_sweep(args)
    if args.workload == "ce-time-sweep":
        return run_ce_time_sweep(args)
    if args.workload == "lattice-sweep":
        return run_lattice_sweep(args)
    if args.workload == "baseline-table":
        return run_baseline_table(args)
    if args.workload == "issue-rate":
        return run_issue_rate(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
