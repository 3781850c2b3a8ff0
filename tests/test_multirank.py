"""The multi-rank (replica) path of bench.py on CPU: two gloo ranks on
127.0.0.1. Each rank owns a disjoint event range, the job's time is the
slowest rank's and its track-steps the sum over ranks, and a replica's results
do not depend on which rank runs it (the CPU oracle stands in for the GPU,
which these ranks do not have)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    import oracle
    from paper_2503_17608_gb300 import workloads as wl

    dist.init_process_group("gloo", rank=rank, world_size=world)
    base = bench.replica_event_base(rank)
    # this rank's replica: two water-cube events of its own
    prob = wl.water_cube_problem(max_events=4)
    prim = np.concatenate([wl.water_cube_primaries(40, event=base + k) for k in range(2)])
    hist, edep = oracle.World(prob).run(prim, n_threads=1)
    steps = int(hist["steps"].sum())
    ms = 10.0 * (rank + 1)
    out[rank] = dict(base=base, steps=steps, edep=float(edep.sum() + hist["escaped"].sum()),
                     max_ms=bench.reduce_over_ranks(ms, "max", dist),
                     sum_steps=bench.reduce_over_ranks(steps, "sum", dist))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_replicas():
    port = free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    assert res[0]["base"] == 0 and res[1]["base"] == 1_000_000
    total = res[0]["steps"] + res[1]["steps"]
    for r in (0, 1):
        assert res[r]["max_ms"] == 20.0            # the slowest rank's time
        assert res[r]["sum_steps"] == total        # every rank's work
        assert res[r]["edep"] == pytest.approx(2 * 40 * 10.0, rel=1e-12)  # each replica conserves energy


def test_replica_results_do_not_depend_on_the_rank():
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2503_17608_gb300 import workloads as wl

    prob = wl.water_cube_problem(max_events=2)
    a = wl.water_cube_primaries(30, event=1_000_000 + 5)
    h1, e1 = oracle.World(prob).run(a, n_threads=1)
    h2, e2 = oracle.World(prob).run(a, n_threads=3)
    np.testing.assert_array_equal(h1["steps"], h2["steps"])
    np.testing.assert_array_equal(e1, e2)


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(3.5, "max") == 3.5
    assert bench.replica_event_base(0) == 0


def test_bench_loop_keys_name_the_library_modes():
    """The bench's loop keys map onto the C ABI's loop modes."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2503_17608_gb300 import binding

    assert bench.LOOP_KEYS["host"] == (binding.LOOP_HOST, False)
    assert bench.LOOP_KEYS["graph"] == (binding.LOOP_GRAPH, False)
    assert bench.LOOP_KEYS["persistent"] == (binding.LOOP_PERSISTENT, False)
    assert bench.LOOP_KEYS["async"] == (binding.LOOP_ASYNC, False)
    assert bench.LOOP_KEYS["async-warps"] == (binding.LOOP_ASYNC, True)


def test_bench_times_each_policy_in_its_loops():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2503_17608_gb300 import workloads as wl

    assert bench.loop_keys_for(wl.SORT_LOCAL, "auto") == ["persistent", "async", "async-warps"]
    assert bench.loop_keys_for(wl.SORT_DATA, "auto") == ["persistent", "async"]
    for pol in (wl.SORT_NONE, wl.SORT_ACTION, wl.SORT_ACTION_TYPE):
        assert bench.loop_keys_for(pol, "auto") == ["persistent"]
        assert bench.loop_keys_for(pol, "async-warps") == ["persistent"]
    assert bench.loop_keys_for(wl.SORT_DATA, "async-warps") == ["async"]
    assert bench.loop_keys_for(wl.SORT_LOCAL, "graph") == ["graph"]


def test_bench_roofline_names_the_timed_kernel():
    sys.path.insert(0, ROOT)
    import bench

    key = ("calorimeter-field-10gev", "local", "async-warps")
    r = bench.roofline_loop(*key, 7959709.0, 5.0, fp64_measured=1.25, sm_mhz=2070.0)
    assert r["kernel"] == "k_loop_async" and r["bound"] == "alu"
    assert r["traffic"] == bench.DRAM_BYTES_PER_LAUNCH[key]
    assert r["peak"] == 1.25 and r["frac"] == r["achieved"] / r["peak"]
    fp = bench.FP64_FLOP_PER_STEP.get(key, bench.FP64_FLOP_PER_STEP[key[:2]])
    assert abs(r["achieved"] - fp * 7959709.0 / 5e-3 / 1e12) < 1e-12
    # FP64 pipe: warp instructions x 64 cycles over 4 sub-partitions x 152 SMs x the clock
    wi = bench.FP64_WARP_INSTR_PER_STEP[key]
    assert abs(r["fp64_pipe"]["busy_frac"] - wi * 7959709.0 * 64 / (5e-3 * 4 * 152 * 2.07e9)) < 1e-12
    # without a measured peak the derived one is used
    assert bench.roofline_loop(*key, 1.0, 1.0)["peak"] == bench.FP64_PEAK_TFLOPS
    # the per-warp kernel was captured whole on both calorimeters; other kernels
    # were not: no traffic figure
    k1 = ("calorimeter-1gev", "local", "async-warps")
    assert bench.roofline_loop(*k1, 1.0, 1.0)["traffic"] == bench.DRAM_BYTES_PER_LAUNCH[k1]
    assert bench.roofline_loop("calorimeter-1gev", "local", "persistent", 1.0, 1.0)["traffic"] is None
    assert bench.roofline_loop("calorimeter-1gev", "local", "async", 1.0, 1.0)["traffic"] is None
    assert bench.roofline_loop("calorimeter-1gev", "local", "persistent", 1.0, 1.0)["kernel"] == "k_loop_local"
    assert bench.roofline_loop("calorimeter-1gev", "none", "persistent", 1.0, 1.0)["kernel"] == "k_loop"
    # a reduced workload carries no traffic figure (the captures were of the full one)
    assert bench.roofline_loop("calorimeter-1gev", "local", "async", 1.0, 1.0, full_size=False)["traffic"] is None
