"""Benchmark: track-steps/s of the step-based transport loop on one GB300.

A "step" of this benchmark is one full transport job: every primary of the
workload queued from device memory and transported until no track is alive
or queued (all step iterations: initializer, step limit, partition,
propagation, interactions, secondaries, tallies). ``value`` is track-steps
per second over K such jobs with the primaries already resident in HBM;
``e2e`` is the same through the host-pointer C ABI with the primaries copied
from pinned host memory and the tallies copied back inside the timed region.

Default workload: the lead/liquid-argon sampling calorimeter, 1,000 x 1 GeV
electrons, 65,536 slots, no field; run with sorting on (partition by particle
type and action) and off.

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
UNIT = "track-steps/s"


def make_workload(name: str):
    if name == "calorimeter-1gev":
        prob, prim = wl.calorimeter_1gev(1000)
        desc = dict(workload="Pb/LAr calorimeter, 1000 x 1 GeV e-, no field", primaries=1000, energy_MeV=1000.0,
                    slots=prob.n_slots, layers=prob.n_layers_total, field_T=0.0)
    elif name == "calorimeter-field-10gev":
        prob, prim = wl.calorimeter_field_10gev(10000)
        desc = dict(workload="Pb/LAr calorimeter in 4 T, 10000 x 10 GeV e-", primaries=10000, energy_MeV=1e4,
                    slots=prob.n_slots, layers=prob.n_layers_total, field_T=4.0)
    elif name == "water-cube-10mev":
        prob, prim = wl.water_cube_problem(), wl.water_cube_primaries()
        desc = dict(workload="water cube, 2000 x 10 MeV photons", primaries=2000, energy_MeV=10.0,
                    slots=prob.n_slots, layers=1, field_T=0.0)
    else:
        raise SystemExit(f"unknown workload {name}")
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
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

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
        for ln in self.lines:
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
    prob, prim, desc = make_workload(args.workload)
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


# ---------------------------------------------------------------- GPU
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

    prob, prim, desc = make_workload(args.workload)
    n = len(prim)
    cprim = binding.to_c_primaries(prim)
    dev_prim = torch.from_numpy(cprim.view(np.uint8).copy()).cuda()
    pinned = torch.empty(cprim.nbytes, dtype=torch.uint8, pin_memory=True)
    pinned_np = pinned.numpy().view(binding.PRIMARY_C)
    pinned_np[:] = cprim
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    policies = [binding_policy(p) for p in args.policies.split(",")]
    headline = binding_policy(args.policy)
    if headline not in policies:
        policies.insert(0, headline)
    use_graph = not args.no_graph
    base_event = rank * 1_000_000

    results = {}
    clocks = None
    for pol in policies:
        ctx = binding.Context(prob.replace(sort_policy=pol, max_events=1), stream=stream.cuda_stream)
        ev = [base_event]

        def job():
            e = ev[0]
            ev[0] += 1
            ctx.reset_event(e)
            ctx.add_primaries_device(e, dev_prim.data_ptr(), n)
            ctx.run_events(use_graph=use_graph)

        for _ in range(args.warmup):
            flush.zero_()
            job()
        s0 = ctx.stats()["steps_total"]
        barrier()
        sampler = ClockSampler(local) if pol == headline else None
        if sampler:
            sampler.__enter__()
        t_start = torch.cuda.Event(enable_timing=True)
        t_stop = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for _ in range(args.steps):
            flush.zero_()
            job()
        t_stop.record(stream)
        barrier()
        if sampler:
            sampler.__exit__()
            clocks = sampler.summary()
        ms = t_start.elapsed_time(t_stop)
        steps = ctx.stats()["steps_total"] - s0
        ms_t = torch.tensor([ms], device="cuda")
        st_t = torch.tensor([float(steps)], device="cuda")
        if dist is not None:
            dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
            dist.all_reduce(st_t, op=dist.ReduceOp.SUM)
        results[pol] = dict(ms=ms_t.item(), steps=st_t.item(), ctx=ctx)

    # end-to-end through the public host-pointer API (headline policy)
    ctx = results[headline]["ctx"]
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
        ctx.run_events(use_graph=use_graph)
        tally, esc = ctx.read_tallies(ev_e2e)
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e_ms += (t1 - t0) * 1e3
            e2e_steps += ctx.stats()["steps_total"] - s0
        ev_e2e += 1
    e2e_t = torch.tensor([e2e_ms], device="cuda")
    e2e_s = torch.tensor([float(e2e_steps)], device="cuda")
    if dist is not None:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
        dist.all_reduce(e2e_s, op=dist.ReduceOp.SUM)

    # per-kernel device time (plain host loop with CUDA events around each launch)
    kt = None
    if not args.no_kernel_timing:
        kctx = binding.Context(prob.replace(sort_policy=headline, max_events=1), stream=stream.cuda_stream)
        kctx.reset_event(7)
        kctx.add_primaries_device(7, dev_prim.data_ptr(), n)
        kctx.run_events(use_graph=False)
        kctx.enable_kernel_timing(True)
        s0 = kctx.stats()
        kctx.reset_event(8)
        kctx.add_primaries_device(8, dev_prim.data_ptr(), n)
        kctx.run_events(use_graph=False)
        s1 = kctx.stats()
        kt = dict(kernels=kctx.kernel_timing(), steps=s1["steps_total"] - s0["steps_total"],
                  iterations=s1["iteration"] - s0["iteration"])
        kctx.close()

    if rank != 0:
        return
    h = results[headline]
    value = h["steps"] / (h["ms"] / 1e3)
    by_policy = {binding_name(p): dict(value=r["steps"] / (r["ms"] / 1e3), ms_per_step=r["ms"] / args.steps,
                                       track_steps_per_job=r["steps"] / args.steps / world)
                 for p, r in results.items()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": h["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(desc, sort_policy=binding_name(headline), graph=use_graph,
                       parallelism=f"replicas x{world} (independent events per rank)",
                       l2="512 MiB buffer written between timed jobs"),
        "sorted_vs_unsorted": by_policy,
        "e2e": {"value": e2e_s.item() / (e2e_t.item() / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(cprim.nbytes),
                "d2h_bytes_per_step": int(8 * (len(tally) + 1))},
        "clocks": clocks,
    }
    if kt is not None:
        line["kernel_timing"] = summarize_kernels(kt)
        line["gpu_launches"] = int(sum(v["launches"] for v in kt["kernels"].values()) * args.steps)
        line["roofline"] = roofline(kt, args)
    if not args.skip_cpu_baseline and world == 1:
        rate, cores, reps, nsample, dt = cpu_oracle_rate(prob, prim, min_seconds=args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"full workload ({nsample} primaries) x {reps} in {dt:.1f} s"}
    print(json.dumps(line), flush=True)
    for r in results.values():
        r["ctx"].close()
    if dist is not None:
        dist.destroy_process_group()


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


def roofline(kt, args):
    peaks, kind = load_peaks()
    ks = kt["kernels"]
    name, v = max(ks.items(), key=lambda kv: kv[1]["total_ms"])
    avg_s = v["total_ms"] / max(v["launches"], 1) / 1e3
    # algorithmic bytes per unit of the dominant kernel (state read + written once)
    per_unit = KERNEL_BYTES.get(name, 160.0)
    units = kt["steps"] / max(v["launches"], 1)
    achieved = per_unit * units / avg_s / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": None, "peak_kind": kind,
            "bytes_per_unit": per_unit, "unit_kind": "track-step"}


# Algorithmic bytes per track-step each kernel must move at minimum (state
# fields read + written once); see the design notes for the accounting.
KERNEL_BYTES = {
    "pre_step": 118.0,
    "along_charged": 100.0,
    "along_neutral": 80.0,
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="calorimeter-1gev",
                    choices=["calorimeter-1gev", "calorimeter-field-10gev", "water-cube-10mev"])
    ap.add_argument("--policy", default="action_type", choices=list(wl.SORT_NAMES))
    ap.add_argument("--policies", default="action_type,action,none")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-kernel-timing", action="store_true")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=3.0)
    ap.add_argument("--reference-primaries", type=int, default=0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
