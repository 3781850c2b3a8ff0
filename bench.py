"""Benchmark: track-steps/s of the step-based transport loop on one GB300.

A "step" of this benchmark is one full transport job: every primary of the
workload queued from device memory and transported until no track is alive
or queued (all step iterations: initializer, step limit, partition,
propagation, interactions, secondaries, tallies). ``value`` is track-steps
per second over K such jobs with the primaries already resident in HBM;
``e2e`` is the same through the host-pointer C ABI with the primaries copied
from pinned host memory and the tallies copied back inside the timed region.

Default workload: the lead/liquid-argon sampling calorimeter in a uniform
4 T field along z, 10,000 x 10 GeV electrons over a 10 cm x 10 cm patch of
the front face, 2^20 track slots; run with every sort policy (none, by
action, by action and particle type, charge partition of the data, block-
local grouping). The 1 GeV calorimeter without field, batched offload
events, event-per-stream and Poisson-arrival serving are reported beside it.

--impl reference times the CPU oracle (the plain history-based transport)
on the host cores on a bounded sample of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2503_17608_gb300 import workloads as wl  # noqa: E402

METRIC = "track-steps/s on 1 GB300, sorted vs unsorted; p50/p99 event latency served"
# loop keys of the bench: (celer loop mode, per-warp scheduling of the asynchronous loop)
LOOP_KEYS = {"host": (0, False), "graph": (1, False), "persistent": (2, False), "async": (3, False),
             "async-warps": (3, True)}
UNIT = "track-steps/s"


def make_workload(name: str, primaries: int = 0, slots: int = 0):
    """The named workload; primaries / slots override its sizes (smaller
    cases of the same shape, e.g. for profiler captures)."""
    if name == "calorimeter-1gev":
        n = primaries or 1000
        prob, prim = wl.calorimeter_1gev(n)
        desc = dict(workload=f"Pb/LAr calorimeter, {n} x 1 GeV e-, no field", primaries=n, energy_MeV=1000.0,
                    layers=prob.n_layers_total, field_T=0.0)
    elif name == "calorimeter-field-10gev":
        n = primaries or 10000
        prob, prim = wl.calorimeter_field_10gev(n)
        desc = dict(workload=f"Pb/LAr calorimeter in 4 T, {n} x 10 GeV e-", primaries=n, energy_MeV=1e4,
                    layers=prob.n_layers_total, field_T=4.0)
    elif name == "water-cube-10mev":
        n = primaries or 2000
        prob, prim = wl.water_cube_problem(), wl.water_cube_primaries(n)
        desc = dict(workload=f"water cube, {n} x 10 MeV photons", primaries=n, energy_MeV=10.0, layers=1, field_T=0.0)
    else:
        raise SystemExit(f"unknown workload {name}")
    if slots:
        prob = prob.replace(n_slots=slots)
    desc["slots"] = prob.n_slots
    return prob, prim, desc


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling during the timed region (SM clock, reasons)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []  # (host time, csv line)
        self.window = None

    def __enter__(self):
        """Start sampling every 20 ms and wait (up to 3 s) for the first
        three samples, so that the sampler is live and past its start-up
        queries when the timed region starts."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.monotonic()
            while len(self.lines) < 3 and time.monotonic() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.005)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def region(self, t_begin, t_end):
        """The timed region in host time; samples inside it (plus the first
        one after it, which covers its tail) make the summary."""
        self.window = (t_begin, t_end)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = self.lines
        if self.window is not None:
            b, e = self.window
            inside = [ln for t, ln in rows if b <= t <= e]
            after = [ln for t, ln in rows if t > e][:1]
            rows = inside + after
        else:
            rows = [ln for _, ln in rows]
        for ln in rows:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- oracle (CPU)
def cpu_oracle_rate(prob, prim, min_seconds=2.0, max_primaries=None):
    import oracle

    world = oracle.World(prob)
    cores = len(os.sched_getaffinity(0))
    sample = prim if max_primaries is None else prim[:max_primaries]
    steps = 0
    t0 = time.perf_counter()
    reps = 0
    while True:
        hist, _ = world.run(sample, n_threads=cores, with_edep=False)
        steps += int(hist["steps"].sum())
        reps += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    dt = time.perf_counter() - t0
    return steps / dt, cores, reps, len(sample), dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    prob, prim, desc = make_workload(args.workload, args.primaries, args.slots)
    import oracle

    world = oracle.World(prob)
    cores = len(os.sched_getaffinity(0))
    sample = prim[: args.reference_primaries] if args.reference_primaries else prim
    for _ in range(args.warmup):
        world.run(sample[: max(1, len(sample) // 10)], n_threads=cores, with_edep=False)
    steps = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        hist, _ = world.run(sample, n_threads=cores, with_edep=False)
        steps += int(hist["steps"].sum())
    dt = time.perf_counter() - t0
    value = steps / dt
    sample_desc = f"{len(sample)} of {len(prim)} primaries per step, {args.steps} steps"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(desc, sort_policy="n/a (history-based CPU oracle)"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample_desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- ranks
# Replicas: each rank transports its own events (no data-path exchange, the
# histories are independent and the random streams are keyed by event);
# only the timing is combined over the ranks.
EVENTS_PER_RANK = 1_000_000


def replica_event_base(rank: int) -> int:
    """First event id of a rank: the ranks' event ranges are disjoint."""
    return rank * EVENTS_PER_RANK


def reduce_over_ranks(value, op_name, dist=None, device="cpu"):
    """The job-wide figure of a per-rank value: "max" (times: the job ends
    with its slowest rank) or "sum" (track-steps: all ranks' work); the value
    itself without a process group."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op_name == "max" else dist.ReduceOp.SUM)
    return t.item()


# ---------------------------------------------------------------- GPU
def loop_keys_for(policy, loop_arg):
    """Loops timed for a policy: the one named (the asynchronous loop only for
    the block-pass policies, its per-warp schedule only for local), else the
    persistent loop and, for the block-pass policies, the asynchronous one
    (block passes, and for local per-warp scheduling too)."""
    block_pass = (wl.SORT_LOCAL, wl.SORT_DATA)
    if loop_arg != "auto":
        key = loop_arg
        if key.startswith("async") and policy not in block_pass:
            key = "persistent"  # the policy comparison runs every policy
        if key == "async-warps" and policy != wl.SORT_LOCAL:
            key = "async"
        return [key]
    keys = ["persistent"]
    if policy in block_pass:
        keys.append("async")
    if policy == wl.SORT_LOCAL:
        keys.append("async-warps")
    return keys


def run_ours(args):
    import torch

    from paper_2503_17608_gb300 import binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def reduce(v, op):
        return reduce_over_ranks(v, op, dist, device="cuda")

    MAX, SUM = "max", "sum"

    prob, prim, desc = make_workload(args.workload, args.primaries, args.slots)
    n = len(prim)
    # the device's FP64 throughput (the ALU roofline's peak), measured here
    fp64_tflops = None
    if not args.no_fp64_probe:
        fp64_tflops = max(binding.debug_fp64_rate()[0] for _ in range(3))
    cprim = binding.to_c_primaries(prim)
    dev_prim = torch.from_numpy(cprim.view(np.uint8).copy()).cuda()
    pinned = torch.empty(cprim.nbytes, dtype=torch.uint8, pin_memory=True)
    pinned_np = pinned.numpy().view(binding.PRIMARY_C)
    pinned_np[:] = cprim
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    policies = [binding_policy(p) for p in args.policies.split(",") if p]
    auto = args.policy == "auto"
    headline = None if auto else binding_policy(args.policy)
    if headline is not None and headline not in policies:
        policies.insert(0, headline)
    base_event = replica_event_base(rank)
    block_pass = (wl.SORT_LOCAL, wl.SORT_DATA)

    def loops_for(pol):
        return loop_keys_for(pol, args.loop)

    def timed_jobs(pol, key, split, steps, warmup, sample_clocks=False):
        """K whole jobs, primaries resident on the device; returns ms, steps, per-job ms."""
        mode, warps = LOOP_KEYS[key]
        ctx = binding.Context(prob.replace(sort_policy=pol, max_events=1, split_actions=int(split)),
                              stream=stream.cuda_stream)
        ctx.set_async_warps(warps)
        ev = [base_event]

        def job():
            e = ev[0]
            ev[0] += 1
            ctx.reset_event(e)
            ctx.add_primaries_device(e, dev_prim.data_ptr(), n)
            ctx.run_events(mode)

        sampler = ClockSampler(local) if sample_clocks else None
        if sampler:
            sampler.__enter__()
        for _ in range(warmup):
            flush.zero_()
            job()
        s0 = ctx.stats()["steps_total"]
        barrier()
        h_begin = time.monotonic()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        stops = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        t_start = torch.cuda.Event(enable_timing=True)
        t_stop = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for k in range(steps):
            flush.zero_()
            starts[k].record(stream)
            job()
            stops[k].record(stream)
        t_stop.record(stream)
        barrier()
        h_end = time.monotonic()
        clocks = None
        if sampler:
            time.sleep(0.05)  # let the sample after the region arrive
            sampler.__exit__()
            sampler.region(h_begin, h_end)
            clocks = sampler.summary()
        region_ms = t_start.elapsed_time(t_stop)  # includes the L2 flushes between jobs
        per_job = [a.elapsed_time(b) for a, b in zip(starts, stops)]
        steps_done = ctx.stats()["steps_total"] - s0
        # the work's time: the K jobs' own CUDA-event intervals (the flushes
        # between them are not part of the work), max over ranks
        return ctx, dict(ms=reduce(sum(per_job), MAX), region_ms=reduce(region_ms, MAX), steps=reduce(steps_done, SUM),
                         job_ms=per_job, clocks=clocks)

    # every (policy, loop) pair is timed the same way; the headline is the
    # fastest pair (of the named policy, if one is named): what the autotuner
    # would pick for this workload
    results = {}
    ctxs = {}
    for pol in policies:
        for key in loops_for(pol):
            ctx, r = timed_jobs(pol, key, args.split, args.steps, args.warmup, sample_clocks=True)
            results[(pol, key)] = r
            ctxs[(pol, key)] = ctx
    pairs = [k for k in results if auto or k[0] == headline]
    headline, loop = max(pairs, key=lambda k: results[k]["steps"] / results[k]["ms"])
    clocks = results[(headline, loop)]["clocks"]
    head_ctx = ctxs.pop((headline, loop))
    for ctx in ctxs.values():
        ctx.close()

    loop_modes = {}
    if not args.no_loop_compare:
        for name, key, split in (("host_per_action", "host", True),
                                 ("graph_per_action", "graph", True),
                                 ("graph_per_phase", "graph", False),
                                 ("persistent", "persistent", False),
                                 ("async", "async", False),
                                 ("async_warps", "async-warps", False)):
            if key.startswith("async") and headline not in block_pass:
                continue
            if key == "async-warps" and headline != wl.SORT_LOCAL:
                continue
            ctx, r = timed_jobs(headline, key, split, max(2, args.steps // 2), 2)
            ctx.close()
            loop_modes[name] = dict(value=r["steps"] / (r["ms"] / 1e3), ms_per_step=r["ms"] / max(2, args.steps // 2))

    # end-to-end through the public host-pointer API (headline policy and loop)
    ctx = head_ctx
    tally = np.zeros(ctx.n_bins)
    e2e_ms = 0.0
    e2e_steps = 0
    ev_e2e = base_event + 500_000
    for k in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        s0 = ctx.stats()["steps_total"]
        t0 = time.perf_counter()
        ctx.reset_event(ev_e2e)
        ctx.add_primaries(ev_e2e, pinned_np)
        ctx.run_events(LOOP_KEYS[loop][0])
        tally, esc = ctx.read_tallies(ev_e2e)
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e_ms += (t1 - t0) * 1e3
            e2e_steps += ctx.stats()["steps_total"] - s0
        ev_e2e += 1
    prof = ctx.loop_profile() if loop == "persistent" else None
    e2e_ms = reduce(e2e_ms, MAX)
    e2e_steps = reduce(e2e_steps, SUM)
    iterations = ctx.stats()["iteration"]

    # per-action kernel device time (host loop, one launch per action, CUDA events around each)
    kt = None
    if not args.no_kernel_timing:
        kctx = binding.Context(prob.replace(sort_policy=headline, max_events=1, split_actions=1),
                               stream=stream.cuda_stream)
        kctx.reset_event(7)
        kctx.add_primaries_device(7, dev_prim.data_ptr(), n)
        kctx.run_events(binding.LOOP_HOST)
        kctx.enable_kernel_timing(True)
        s0 = kctx.stats()
        kctx.reset_event(8)
        kctx.add_primaries_device(8, dev_prim.data_ptr(), n)
        kctx.run_events(binding.LOOP_HOST)
        s1 = kctx.stats()
        kt = dict(kernels=kctx.kernel_timing(), steps=s1["steps_total"] - s0["steps_total"],
                  iterations=s1["iteration"] - s0["iteration"])
        kctx.close()

    if rank != 0:
        return
    h = results[(headline, loop)]
    value = h["steps"] / (h["ms"] / 1e3)
    steps_per_job = h["steps"] / args.steps / world
    # per policy, in the persistent loop (the sorted vs unsorted comparison),
    # and the block-pass policies again in the asynchronous loop
    by_policy = {binding_name(p) + ("" if m == "persistent" else f" ({m} loop)"):
                 dict(value=r["steps"] / (r["ms"] / 1e3), ms_per_step=r["ms"] / args.steps,
                      track_steps_per_job=r["steps"] / args.steps / world)
                 for (p, m), r in results.items()}
    # per job: primaries push, run start, (block-pass policies: per-block
    # vacancy scan; asynchronous loop: buffer entry states), loop kernel
    if loop.startswith("async"):
        launches_per_job = 5
    elif loop == "persistent":
        launches_per_job = 4 if headline in block_pass else 3
    else:
        launches_per_job = None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": h["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "timed_region_ms": h["region_ms"],
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(desc, sort_policy=binding_name(headline), loop=loop + (" per-action" if args.split else ""),
                       parallelism=f"replicas x{world} (independent events per rank)",
                       l2="512 MiB buffer written between timed jobs (outside the jobs' CUDA-event intervals; timed_region_ms includes it)"),
        "sorted_vs_unsorted": by_policy,
        "loop_modes": loop_modes,
        "e2e": {"value": e2e_steps / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(cprim.nbytes),
                "d2h_bytes_per_step": int(8 * (len(tally) + 1))},
        "clocks": clocks,
    }
    if prof is not None:
        it = max(ctx.stats()["iteration"], 1)
        line["loop_profile_us_per_iteration"] = {
            part: {name: round(c / it / 2.07e3, 3) for name, c in vals.items()} for part, vals in prof.items()}
    job_ms = statistics.median(h["job_ms"])
    line["roofline"] = roofline_loop(args.workload, binding_name(headline), loop, steps_per_job, job_ms,
                                     full_size=not (args.primaries or args.slots), fp64_measured=fp64_tflops,
                                     sm_mhz=(clocks or {}).get("sm_mhz"),
                                     sms=torch.cuda.get_device_properties(local).multi_processor_count)
    if launches_per_job:
        line["gpu_launches"] = int(launches_per_job * args.steps)
    if kt is not None:
        line["kernel_timing"] = summarize_kernels(kt)
        if not launches_per_job:
            per_job = sum(v["launches"] for v in kt["kernels"].values())
            line["gpu_launches"] = int((per_job + 1) * args.steps)
    if not args.no_extras and world == 1:
        line["other_workloads"] = run_extras(args, binding, stream, flush)
    if not args.skip_cpu_baseline and world == 1:
        rate, cores, reps, nsample, dt = cpu_oracle_rate(prob, prim, min_seconds=args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"full workload ({nsample} primaries) x {reps} in {dt:.1f} s"}
    print(json.dumps(line), flush=True)
    head_ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def run_extras(args, binding, stream, flush):
    """The other workloads of the benchmark suite, reported beside the headline:
    the 4 T / 10 GeV calorimeter at 2^20 slots (all sort policies), 256
    offload events batched in one loop (autotuned) vs 256 sequential runs, and
    Poisson-arrival serving vs the one-event-at-a-time loop."""
    import torch

    out = {}
    # --- 1,000 x 1 GeV e-, no field, 65,536 slots: every policy in the
    # persistent loop, the block-pass policies in the asynchronous one
    prob1, prim1, desc1 = make_workload("calorimeter-1gev")
    c1 = binding.to_c_primaries(prim1)
    dev1 = torch.from_numpy(c1.view(np.uint8).copy()).cuda()
    pol = {}
    runs = [(name, binding.LOOP_PERSISTENT) for name in ("action_type", "action", "none", "data", "local")]
    runs += [("data", binding.LOOP_ASYNC), ("local", binding.LOOP_ASYNC), ("local", "async-warps")]
    for name, mode in runs:
        ctx = binding.Context(prob1.replace(sort_policy=wl.SORT_NAMES[name], max_events=1), stream=stream.cuda_stream)
        label = name if mode == binding.LOOP_PERSISTENT else f"{name} ({mode if isinstance(mode, str) else 'async'} loop)"
        ctx.set_async_warps(mode == "async-warps")
        if mode == "async-warps":
            mode = binding.LOOP_ASYNC
        times, steps = [], 0
        for rep in range(3 + 2 * args.extra_steps):
            flush.zero_()
            ctx.reset_event(rep)
            s0 = ctx.stats()["steps_total"]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.add_primaries_device(rep, dev1.data_ptr(), len(c1))
            ctx.run_events(mode)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep >= 3:
                times.append(e0.elapsed_time(e1))
                steps += ctx.stats()["steps_total"] - s0
        it = ctx.stats()["iteration"]
        ctx.close()
        ms = sum(times)
        pol[label] = dict(value=steps / (ms / 1e3), ms_per_job=ms / len(times), track_steps_per_job=steps / len(times),
                          iterations_per_job=it / (3 + 2 * args.extra_steps))
    out["calorimeter_1gev"] = dict(desc1, sorted_vs_unsorted=pol)
    prob2, prim2, desc2 = make_workload("calorimeter-field-10gev")
    c2 = binding.to_c_primaries(prim2)
    dev2 = torch.from_numpy(c2.view(np.uint8).copy()).cuda()

    # --- Runge-Kutta field propagation with a substep cap (paper Sec. 3.3, Fig. 2):
    # the 4 T workload with substeps of at most 0.1 rad, caps of 10^9 (none),
    # 1000 and 10 substeps per step, block-local policy
    rk = {}
    for cap in (1 << 30, 1000, 10):
        ctx = binding.Context(prob2.replace(sort_policy=wl.SORT_LOCAL, max_events=1, field_substep_cap=cap),
                              stream=stream.cuda_stream)
        times, steps, iters = [], 0, 0
        for rep in range(1 + args.extra_steps):
            flush.zero_()
            ctx.reset_event(rep)
            s0 = ctx.stats()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.add_primaries_device(rep, dev2.data_ptr(), len(c2))
            ctx.run_events(binding.LOOP_PERSISTENT)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep >= 1:
                s1 = ctx.stats()
                times.append(e0.elapsed_time(e1))
                steps += s1["steps_total"] - s0["steps_total"]
                iters += s1["iteration"] - s0["iteration"]
        ctx.close()
        nrep = len(times)
        rk["no_cap" if cap == 1 << 30 else f"cap_{cap}"] = dict(
            value=steps / (sum(times) / 1e3), ms_per_job=sum(times) / nrep, track_steps_per_job=steps / nrep,
            iterations_per_job=iters / nrep)
    out["field_runge_kutta_substep_cap"] = dict(workload=desc2["workload"], substep_turn_rad=0.1, runs=rk)

    # --- parent-slot reuse (paper Sec. 3.2) on the 1 GeV calorimeter, per policy
    reuse = {}
    for name in ("none", "data", "local"):
        row = {}
        for on in (False, True):
            ctx = binding.Context(prob1.replace(sort_policy=wl.SORT_NAMES[name], max_events=1), stream=stream.cuda_stream)
            ctx.set_parent_reuse(on)
            times, steps = [], 0
            for rep in range(3 + args.extra_steps):
                flush.zero_()
                ctx.reset_event(rep)
                s0 = ctx.stats()["steps_total"]
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.add_primaries_device(rep, dev1.data_ptr(), len(c1))
                ctx.run_events(binding.LOOP_PERSISTENT)
                e1.record(stream)
                torch.cuda.synchronize()
                if rep >= 3:
                    times.append(e0.elapsed_time(e1))
                    steps += ctx.stats()["steps_total"] - s0
            ctx.close()
            row["reuse" if on else "queued"] = steps / (sum(times) / 1e3)
        reuse[name] = row
    out["parent_slot_reuse"] = dict(workload=desc1["workload"], track_steps_per_s=reuse)

    # --- 256 offload events: autotune on a sample, then all in one loop vs one by one
    events = wl.offload_events(256)
    prim3 = wl.concat_primaries(events)
    base3 = wl.calorimeter_problem(1 << 20, Bz=4.0, max_events=256)
    sample = wl.concat_primaries(events[:24])
    best, trials = binding.autotune(base3, sample, [1 << 18, 1 << 19, 1 << 20, 1 << 21], [128, 256, 512],
                                    [wl.SORT_NONE, wl.SORT_ACTION, wl.SORT_ACTION_TYPE, wl.SORT_LOCAL, wl.SORT_DATA],
                                    [binding.LOOP_PERSISTENT, binding.LOOP_GRAPH, binding.LOOP_ASYNC],
                                    stream=stream.cuda_stream)
    tuned = base3.replace(n_slots=best["n_slots"], block_size=best["block_size"], sort_policy=best["sort_policy"],
                          init_capacity=max(8 * best["n_slots"], 1 << 22))
    mode = best["mode"]
    ctx = binding.Context(tuned, stream=stream.cuda_stream)
    ctx.set_async_warps(best["async_warps"])
    ctx.add_events(prim3)  # warm-up pass
    ctx.run_events(mode)
    for e in range(256):
        ctx.reset_event(e)
    flush.zero_()
    torch.cuda.synchronize()
    s0 = ctx.stats()["steps_total"]
    t0 = time.perf_counter()
    ctx.add_events(prim3)
    ctx.run_events(mode)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    steps_batch = ctx.stats()["steps_total"] - s0
    batched_tallies = [ctx.read_tallies(e) for e in range(256)]
    ctx.close()
    ctx = binding.Context(tuned.replace(max_events=1), stream=stream.cuda_stream)
    ctx.set_async_warps(best["async_warps"])
    s0 = ctx.stats()["steps_total"]
    t0 = time.perf_counter()
    seq_tallies = []
    for e, ev in enumerate(events):
        ctx.reset_event(e)
        ctx.add_primaries(e, ev)
        ctx.run_events(mode)
        seq_tallies.append(ctx.read_tallies(e))
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    steps_seq = ctx.stats()["steps_total"] - s0
    ctx.close()
    max_rel = max(float(np.max(np.abs(b[0] - q[0]) / np.maximum(np.abs(q[0]), 1e-300))) for b, q in
                  zip(batched_tallies, seq_tallies))
    out["offload_batched_256"] = dict(
        events=256, primaries=int(len(prim3)), autotuned=dict(best, trials=len(trials)),
        batched=dict(value=steps_batch / t_batch, wall_s=t_batch, track_steps=int(steps_batch),
                     events_per_s=256 / t_batch),
        sequential=dict(value=steps_seq / t_seq, wall_s=t_seq, track_steps=int(steps_seq), events_per_s=256 / t_seq),
        speedup=t_seq / t_batch, max_rel_tally_diff_batched_vs_sequential=max_rel)
    out["event_per_stream"] = event_per_stream(binding, tuned, events[:64], seq_tallies[:64], flush)

    # --- serving: Poisson arrivals of offload events. The configured stream
    # (2,000 events/s for 60 s) with continuous batching; then the capacity of
    # the one-event-at-a-time loop (offered the same stream for a few seconds,
    # its queue grows, so its sustained rate is its capacity), and both loops
    # at 0.5x and 0.8x of that capacity, where both queues are stable and the
    # latency percentiles describe a steady state
    sprob = tuned.replace(max_events=4096)
    cb_mode = binding.LOOP_ASYNC if sprob.sort_policy in (wl.SORT_LOCAL, wl.SORT_DATA) else binding.LOOP_PERSISTENT

    def serve_run(rate_hz, seconds, mode, max_in_flight=0):
        arrivals = wl.poisson_arrivals(rate_hz, seconds)
        sev = wl.offload_events(len(arrivals), first_event=0)
        reqs = [(float(t), i, e) for i, (t, e) in enumerate(zip(arrivals, sev))]
        ctx = binding.Context(sprob, stream=stream.cuda_stream)
        ctx.set_async_warps(best["async_warps"])
        res, summ, _ = ctx.serve(reqs, mode=mode, chunk_iterations=args.serve_chunk,
                                 stop_admitting_s=seconds + 0.5, max_in_flight=max_in_flight)
        ctx.close()
        done = res["done_s"] >= 0
        lat = (res["done_s"] - res["arrival_s"])[done]
        return dict(
            mode={binding.LOOP_PERSISTENT: "persistent", binding.LOOP_ASYNC: "async"}[mode],
            offered_events=len(reqs), offered_rate=len(reqs) / seconds, completed=int(done.sum()),
            sustained_rate=float(done.sum() / max(summ["wall_s"], 1e-9)), wall_s=summ["wall_s"],
            track_steps_per_s=summ["track_steps"] / max(summ["wall_s"], 1e-9),
            latency_ms=dict(p50=float(np.percentile(lat, 50) * 1e3), p95=float(np.percentile(lat, 95) * 1e3),
                            p99=float(np.percentile(lat, 99) * 1e3)) if len(lat) else None,
            window_s=seconds)

    served = {}
    served["continuous_batching"] = serve_run(args.serve_rate, args.serve_seconds, cb_mode)
    cap = serve_run(args.serve_rate, args.serve_plain_seconds, binding.LOOP_PERSISTENT, max_in_flight=1)
    served["one_event_at_a_time_overloaded"] = cap
    capacity = cap["sustained_rate"]
    stable = {}
    for frac in (0.5, 0.8):
        r = frac * capacity
        stable[f"{frac}x_capacity"] = dict(
            offered_rate_hz=r,
            one_event_at_a_time=serve_run(r, args.serve_stable_seconds, binding.LOOP_PERSISTENT, max_in_flight=1),
            continuous_batching=serve_run(r, args.serve_stable_seconds, cb_mode))
    out["serving"] = dict(rate_hz=args.serve_rate, duration_s=args.serve_seconds, chunk_iterations=args.serve_chunk,
                          sort_policy=binding_name(sprob.sort_policy), one_event_at_a_time_capacity_hz=capacity,
                          stable_queue_comparison=stable, **served)
    return out


def event_per_stream(binding, prob, events, ref_tallies, flush):
    """Event-per-stream mode (paper Sec. 4.1, Fig. 3) with per-iteration hit
    copies (Sec. 3.4): K contexts, each on its own stream with slots/K track
    slots and SMs/K blocks, each stepping one event at a time in the host loop
    and copying its hits to pinned memory after every iteration, against one
    mixed context stepping all events in one track array (persistent loop)."""
    import torch

    n_ev = len(events)
    prim = wl.concat_primaries(events)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    res = {}
    # one mixed track array, all events at once
    stream = torch.cuda.Stream()
    ctx = binding.Context(prob.replace(max_events=n_ev, sort_policy=wl.SORT_LOCAL), stream=stream.cuda_stream)
    ctx.add_events(prim)
    ctx.run_events(binding.LOOP_PERSISTENT)
    for e in range(n_ev):
        ctx.reset_event(e)
    flush.zero_()
    torch.cuda.synchronize()
    s0 = ctx.stats()["steps_total"]
    t0 = time.perf_counter()
    ctx.add_events(prim)
    ctx.run_events(binding.LOOP_PERSISTENT)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    res["mixed_one_array"] = dict(events_per_s=n_ev / dt, value=(ctx.stats()["steps_total"] - s0) / dt)
    ctx.close()

    def run(k_streams, hit_mode):
        ctxs, hits = [], []
        for k in range(k_streams):
            st = torch.cuda.Stream()
            c = binding.Context(prob.replace(n_slots=max(prob.n_slots // k_streams, 1024), max_events=1,
                                             sort_policy=wl.SORT_LOCAL), stream=st.cuda_stream)
            c.set_grid_blocks(max(sms // k_streams, 1))
            h = torch.zeros(c.n_bins, dtype=torch.float64, pin_memory=True)
            c.set_hit_readout(hit_mode, h)
            ctxs.append(c)
            hits.append(h)
        out_t = [None] * n_ev
        steps = [0] * k_streams
        errors = []

        def worker(k):
            try:
                c = ctxs[k]
                s_begin = c.stats()["steps_total"]
                for e in range(k, n_ev, k_streams):
                    c.reset_event(e)
                    c.add_primaries(e, events[e])
                    c.run_events(binding.LOOP_HOST)
                    out_t[e] = c.read_tallies(e)
                steps[k] = c.stats()["steps_total"] - s_begin
            except Exception as exc:  # reported below
                errors.append(repr(exc))

        for c in ctxs:  # warm-up: one event each
            c.reset_event(0)
            c.add_primaries(0, events[0])
            c.run_events(binding.LOOP_HOST)
        flush.zero_()
        torch.cuda.synchronize()
        th = [threading.Thread(target=worker, args=(k,)) for k in range(k_streams)]
        t0 = time.perf_counter()
        for t in th:
            t.start()
        for t in th:
            t.join()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        for c in ctxs:
            c.close()
        if errors:
            return dict(error=errors[0])
        max_rel = max(float(np.max(np.abs(a[0] - b[0]) / np.maximum(np.abs(b[0]), 1e-300)))
                      for a, b in zip(out_t, ref_tallies))
        return dict(events_per_s=n_ev / dt, value=sum(steps) / dt, max_rel_tally_diff_vs_sequential=max_rel)

    for k_streams in (1, 4, 8):
        res[f"streams_{k_streams}_async_hits"] = run(k_streams, 1)
    for k_streams in (4, 8):
        res[f"streams_{k_streams}_sync_hits"] = run(k_streams, 2)
    res["events"] = n_ev
    res["slots_total"] = prob.n_slots
    return res


def binding_policy(name):
    return wl.SORT_NAMES[name]


def binding_name(pol):
    return {v: k for k, v in wl.SORT_NAMES.items()}[pol]


def summarize_kernels(kt):
    ks = kt["kernels"]
    total = sum(v["total_ms"] for v in ks.values()) or 1.0
    out = {}
    for name, v in sorted(ks.items(), key=lambda kv: -kv[1]["total_ms"]):
        if v["launches"] == 0:
            continue
        out[name] = dict(launches=v["launches"], total_ms=round(v["total_ms"], 4),
                         avg_us=round(1e3 * v["total_ms"] / v["launches"], 3), share=round(v["total_ms"] / total, 4))
    return dict(per_kernel=out, track_steps=kt["steps"], iterations=kt["iterations"])


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


# Per track-step figures of the whole step loop (all phases of an iteration):
# algorithmic state bytes (state read and written back once per step, without
# secondaries or scratch) and thread-level FP64 operations
# (2 x DFMA + DADD + DMUL) counted by ncu on the loop kernels (the ncu
# summaries under profiles/, one per kernel and workload). DRAM bytes per
# launch come from one-pass full-size captures of the per-warp kernel on the
# two calorimeters; other kernels report no traffic. Keys: (workload, policy), and
# (workload, policy, loop) for the asynchronous loop kernel.
BYTES_PER_STEP = 160.0
FP64_FLOP_PER_STEP = {("calorimeter-1gev", "none"): 97.0, ("calorimeter-1gev", "action"): 97.0,
                      ("calorimeter-1gev", "action_type"): 97.0, ("calorimeter-1gev", "data"): 86.4,
                      ("calorimeter-1gev", "local"): 86.4, ("calorimeter-1gev", "local", "async-warps"): 86.5,
                      ("calorimeter-field-10gev", "none"): 95.7, ("calorimeter-field-10gev", "action"): 95.7,
                      ("calorimeter-field-10gev", "action_type"): 95.7, ("calorimeter-field-10gev", "data"): 92.5,
                      ("calorimeter-field-10gev", "local"): 92.5,
                      # the 4 T workload's counts come from its smaller case (2,500
                      # primaries, 2^18 slots; the op counters take 3 passes)
                      ("calorimeter-field-10gev", "local", "async-warps"): 92.5,
                      # water cube: k_loop (none; action and action_type run the same
                      # kernel and counted the same on the calorimeters) and the others
                      ("water-cube-10mev", "none"): 290.5, ("water-cube-10mev", "action"): 290.5,
                      ("water-cube-10mev", "action_type"): 290.5, ("water-cube-10mev", None): 286.7}
DRAM_BYTES_PER_LAUNCH = {("calorimeter-field-10gev", "local", "async-warps"): 49.74e6,
                         ("calorimeter-1gev", "local", "async-warps"): 3.39e6}
# FP64 warp instructions per track-step (sm__inst_executed_pipe_fp64 / track-steps)
# of the loop kernel's one-launch ncu captures: an FP64 warp instruction holds
# its sub-partition's FP64 pipe for 64 cycles whatever its active lanes, so
# these set how busy the FP64 pipe is at a measured track-step rate.
FP64_WARP_INSTR_PER_STEP = {("calorimeter-field-10gev", "local", "async-warps"): 3.36,
                            ("calorimeter-1gev", "local", "async-warps"): 8.04}
FP64_PIPE_CYCLES_PER_WARP_INSTR = 64.0
# FP64 peak of GB300 derived from its unit counts: 2 DFMA per SM-cycle
# (ncu peak_sustained) x 152 SMs x 2.07 GHz x 2 flop
FP64_PEAK_TFLOPS = 2 * 152 * 2.07e9 * 2 / 1e12


def roofline_loop(workload, policy, loop, steps_per_job, job_ms, full_size=True, fp64_measured=None, sm_mhz=None,
                  sms=152):
    """Roofline of the dominant kernel, the step-loop kernel (one launch per
    job): FP64 ALU bound against the FP64 throughput measured on this device
    in the same run (the derived peak beside it), with the FP64 pipe's busy
    fraction and the HBM fraction."""
    peaks, kind = load_peaks()
    t = job_ms / 1e3
    key = (workload, policy) if not loop.startswith("async") else (workload, policy, loop)
    fpstep = FP64_FLOP_PER_STEP.get(key, FP64_FLOP_PER_STEP.get((workload, policy),
                                                                FP64_FLOP_PER_STEP.get((workload, None), 119.5)))
    flops = fpstep * steps_per_job / t / 1e12
    gbs = BYTES_PER_STEP * steps_per_job / t / 1e9
    if loop.startswith("async"):
        kernel = "k_loop_async"
    else:
        kernel = "k_loop_local" if policy in ("local", "data") else "k_loop"
    peak = fp64_measured if fp64_measured else FP64_PEAK_TFLOPS
    out = {"kernel": kernel, "bound": "alu", "achieved": flops, "peak": peak, "unit": "TFLOP/s",
           "frac": flops / peak, "traffic": DRAM_BYTES_PER_LAUNCH.get(key) if full_size else None,
           "peak_kind": ("measured in this run: FP64 FMA chains on every SM (celer_debug_fp64_rate)"
                         if fp64_measured else "derived: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz"),
           "peak_derived": FP64_PEAK_TFLOPS, "frac_of_derived": flops / FP64_PEAK_TFLOPS,
           "fp64_flop_per_track_step": fpstep,
           "hbm": {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                   "bytes_per_track_step": BYTES_PER_STEP, "peak_kind": kind},
           "launch_ms": job_ms, "track_steps_per_launch": steps_per_job}
    wi = FP64_WARP_INSTR_PER_STEP.get(key) if full_size else None
    if wi is not None:
        clock_hz = (sm_mhz or 2070.0) * 1e6
        busy = wi * steps_per_job * FP64_PIPE_CYCLES_PER_WARP_INSTR / (t * 4 * sms * clock_hz)
        out["fp64_pipe"] = {"warp_instr_per_track_step": wi, "busy_frac": busy,
                            "how": "ncu FP64 warp instructions per track-step x 64 pipe cycles each x track-steps "
                                   "per job / (job time x 4 sub-partitions x SMs x median SM clock)"}
    return out


def run_lane_counters(args):
    """Mean active lanes per instrumented site for every (policy, loop) pair on
    the workload, from the diagnostic build of the library (active-lane
    counters compiled in; its timing is not a benchmark number). Prints one
    JSON line."""
    import torch

    from paper_2503_17608_gb300 import binding, build

    binding.load(build.build(lanes=True))
    torch.cuda.set_device(0)
    prob, prim, desc = make_workload(args.workload, args.primaries, args.slots)
    cprim = binding.to_c_primaries(prim)
    dev_prim = torch.from_numpy(cprim.view(np.uint8).copy()).cuda()
    stream = torch.cuda.current_stream()
    table = {}
    for name in [p for p in args.policies.split(",") if p]:
        pol = wl.SORT_NAMES[name]
        for key in loop_keys_for(pol, args.loop):
            mode, warps = LOOP_KEYS[key]
            ctx = binding.Context(prob.replace(sort_policy=pol, max_events=1), stream=stream.cuda_stream)
            ctx.set_async_warps(warps)
            ctx.reset_event(0)
            ctx.add_primaries_device(0, dev_prim.data_ptr(), len(prim))
            ctx.run_events(mode)  # warm-up job
            torch.cuda.synchronize()
            binding.debug_lane_counts()  # clears
            s0 = ctx.stats()["steps_total"]
            ctx.reset_event(1)
            ctx.add_primaries_device(1, dev_prim.data_ptr(), len(prim))
            ctx.run_events(mode)
            torch.cuda.synchronize()
            counts = binding.debug_lane_counts()
            steps = ctx.stats()["steps_total"] - s0
            ctx.close()
            row = {}
            for site, (v, l, cyc) in counts.items():
                if v == 0:
                    continue
                row[site] = dict(visits=v, mean_lanes=round(l / v, 3), per_track_step=round(v / max(steps, 1), 4))
                if cyc:
                    row[site]["mean_us"] = round(cyc / v / 2070.0, 3)
            table[name + ("" if key == "persistent" else f" ({key} loop)")] = row
    print(json.dumps({"lane_counters": table, "config": desc}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="calorimeter-field-10gev",
                    choices=["calorimeter-1gev", "calorimeter-field-10gev", "water-cube-10mev"])
    ap.add_argument("--policy", default="auto", choices=["auto"] + list(wl.SORT_NAMES))
    ap.add_argument("--split", action="store_true", help="one kernel per action in the host or graph loop")
    ap.add_argument("--primaries", type=int, default=0, help="override the workload's primary count")
    ap.add_argument("--slots", type=int, default=0, help="override the workload's track-slot count")
    ap.add_argument("--policies", default="action_type,action,none,data,local")
    ap.add_argument("--loop", default="auto", choices=["auto"] + list(LOOP_KEYS),
                    help="auto: the persistent loop for every policy, the asynchronous one for local and data, "
                         "and its per-warp scheduling for local")
    ap.add_argument("--no-loop-compare", action="store_true")
    ap.add_argument("--no-kernel-timing", action="store_true")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=3.0)
    ap.add_argument("--reference-primaries", type=int, default=0)
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-fp64-probe", action="store_true", help="use the derived FP64 peak instead of measuring it")
    ap.add_argument("--extra-steps", type=int, default=2)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-plain-seconds", type=float, default=3.0,
                    help="window of the overloaded one-event-at-a-time run that measures its capacity")
    ap.add_argument("--serve-stable-seconds", type=float, default=20.0,
                    help="window of each run at 0.5x and 0.8x of the one-event-at-a-time capacity")
    ap.add_argument("--serve-chunk", type=int, default=8)
    ap.add_argument("--lane-counters", action="store_true",
                    help="print mean active lanes per site and policy from the diagnostic build, then exit")
    args = ap.parse_args()
    if args.lane_counters:
        run_lane_counters(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
