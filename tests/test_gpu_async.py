"""The asynchronous block loop (CELER_LOOP_ASYNC): every block steps its own
slots with no grid barrier and the initializer buffer is a concurrent queue.
A track's draws are keyed by its own id, so every history must equal the
synchronous loops' and the oracle's; only the summation order of the tallies
may differ."""
import numpy as np
import pytest

from paper_2503_17608_gb300 import binding, workloads as wl

from gpu_helpers import assert_conservation, match_fraction, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

# (policy, per-warp scheduling) pairs of the asynchronous loop
SCHEDULES = [(wl.SORT_LOCAL, False), (wl.SORT_LOCAL, True), (wl.SORT_DATA, False)]
SCHED_IDS = ["local-passes", "local-warps", "data-passes"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    binding.load()


def run_async(prob, prim, policy, warps):
    """run_gpu in the asynchronous loop with the given scheduling."""
    prob = prob.replace(sort_policy=policy, history_capacity=len(prim))
    with binding.Context(prob) as ctx:
        ctx.set_async_warps(warps)
        ctx.add_events(prim)
        ctx.run_events(binding.LOOP_ASYNC)
        out = dict(stats=ctx.stats())
        out["hist"], out["edep"] = ctx.read_history(0, len(prim))
        out["tally"] = {e: ctx.read_tallies(e) for e in dict.fromkeys(prim["event"].tolist())}
    return out


def assert_same_histories(a, b, rtol=1e-12):
    np.testing.assert_array_equal(a["hist"]["steps"], b["hist"]["steps"])
    np.testing.assert_array_equal(a["hist"]["secondaries"], b["hist"]["secondaries"])
    np.testing.assert_allclose(a["edep"], b["edep"], rtol=rtol, atol=1e-12)
    np.testing.assert_allclose(a["hist"]["escaped"], b["hist"]["escaped"], rtol=rtol, atol=1e-12)


@pytest.mark.parametrize("policy,warps", SCHEDULES, ids=SCHED_IDS)
def test_water_cube_histories_bit_exact(policy, warps):
    prob = wl.water_cube_problem()
    prim = wl.water_cube_primaries()
    g = run_async(prob, prim, policy, warps)
    o = run_oracle(prob, prim)
    np.testing.assert_array_equal(g["hist"]["steps"], o["hist"]["steps"])
    np.testing.assert_array_equal(g["hist"]["secondaries"], o["hist"]["secondaries"])
    np.testing.assert_allclose(g["edep"], o["edep"], rtol=1e-9, atol=1e-9 * 10.0)
    tally, escaped = g["tally"][0]
    np.testing.assert_allclose(tally, o["edep"].sum(0), rtol=1e-9, atol=1e-6)
    assert escaped == pytest.approx(o["hist"]["escaped"].sum(), rel=1e-9)
    assert_conservation(prim, g["tally"])
    assert g["stats"]["steps_total"] == o["hist"]["steps"].sum()
    assert g["stats"]["alive"] == 0 and g["stats"]["queued"] == 0


@pytest.mark.parametrize("policy,warps", SCHEDULES, ids=SCHED_IDS)
def test_calorimeter_histories_equal_the_synchronous_loop(policy, warps):
    prob, prim = wl.calorimeter_1gev(200)
    a = run_async(prob, prim, policy, warps)
    s = run_gpu(prob, prim, mode=binding.LOOP_PERSISTENT, policy=policy)
    assert_same_histories(a, s)
    assert a["stats"]["steps_total"] == s["stats"]["steps_total"]
    frac, _ = match_fraction(a, run_oracle(prob, prim))
    assert frac == 1.0, frac  # every history matched in every recorded run
    assert_conservation(prim, a["tally"])
    np.testing.assert_allclose(a["tally"][0][0], s["tally"][0][0], rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("policy,warps", SCHEDULES, ids=SCHED_IDS)
def test_field_histories_equal_the_synchronous_loop(policy, warps):
    prob, prim = wl.calorimeter_field_10gev(40, n_slots=1 << 16)
    a = run_async(prob, prim, policy, warps)
    s = run_gpu(prob, prim, mode=binding.LOOP_PERSISTENT, policy=policy)
    assert_same_histories(a, s)
    assert_conservation(prim, a["tally"])


@pytest.mark.parametrize("warps", [False, True])
@pytest.mark.parametrize("n_slots", [1, 7, 1000, 2049])
def test_ragged_slot_counts(n_slots, warps):
    """Fewer slots than blocks (most blocks own none), and partial chunks."""
    prim = wl.water_cube_primaries(150)
    prob = wl.water_cube_problem(n_slots=n_slots, init_capacity=4096)
    g = run_async(prob, prim, wl.SORT_LOCAL, warps)
    o = run_oracle(prob, prim)
    np.testing.assert_array_equal(g["hist"]["steps"], o["hist"]["steps"])
    np.testing.assert_allclose(g["edep"], o["edep"], rtol=1e-9, atol=1e-8)


@pytest.mark.parametrize("policy,warps", SCHEDULES, ids=SCHED_IDS)
def test_small_buffer_defers_without_changing_histories(policy, warps):
    """A 64-entry buffer against a 1 GeV shower: writers find no room and
    defer, readers free entries; the histories are the synchronous loop's."""
    prob, prim = wl.calorimeter_1gev(20)
    prob = prob.replace(n_slots=256, init_capacity=64)
    a = run_async(prob, prim, policy, warps)
    s = run_gpu(prob, prim, mode=binding.LOOP_PERSISTENT, policy=policy)
    assert_same_histories(a, s)
    assert_conservation(prim, a["tally"])


@pytest.mark.parametrize("warps", [False, True])
def test_empty_run(warps):
    prob = wl.water_cube_problem(sort_policy=wl.SORT_LOCAL)
    with binding.Context(prob) as ctx:
        ctx.set_async_warps(warps)
        ctx.run_events(binding.LOOP_ASYNC)
        s = ctx.stats()
        assert s["steps_total"] == 0 and s["alive"] == 0 and s["queued"] == 0


@pytest.mark.parametrize("warps", [False, True])
def test_finishes_runs_begun_by_the_synchronous_loops(warps):
    """Live tracks in slots and entries queued at the start of the run (left
    by budgeted synchronous runs of both block-pass policies): the run's end
    condition counts them, and every history matches the oracle."""
    prob = wl.water_cube_problem(n_slots=1024, history_capacity=2000)
    prim = wl.water_cube_primaries()
    with binding.Context(prob) as ctx:
        ctx.set_async_warps(warps)
        ctx.add_events(prim)
        ctx.set_sort_policy(wl.SORT_DATA)
        ctx.run_iterations(binding.LOOP_PERSISTENT, budget=4)
        ctx.set_sort_policy(wl.SORT_LOCAL)
        ctx.run_iterations(binding.LOOP_GRAPH, budget=3)
        s = ctx.stats()
        assert s["alive"] > 0 and s["queued"] > 0
        ctx.run_events(binding.LOOP_ASYNC)
        s = ctx.stats()
        assert s["alive"] == 0 and s["queued"] == 0
        hist, edep = ctx.read_history(0, len(prim))
        tally = {0: ctx.read_tallies(0)}
    o = run_oracle(prob, prim)
    np.testing.assert_array_equal(hist["steps"], o["hist"]["steps"])
    np.testing.assert_array_equal(hist["secondaries"], o["hist"]["secondaries"])
    np.testing.assert_allclose(edep, o["edep"], rtol=1e-9, atol=1e-9 * 10.0)
    assert_conservation(prim, tally)


def test_synchronous_runs_after_an_asynchronous_one():
    """The vacancy counts the asynchronous loop leaves behind serve the next
    runs of every policy on the same context (one event per run)."""
    prob = wl.water_cube_problem(n_slots=2048, history_capacity=8000)
    batches = []
    for k in range(4):
        b = wl.water_cube_primaries()
        b["event"][:] = k
        batches.append(b)
    runs = ((wl.SORT_LOCAL, binding.LOOP_ASYNC), (wl.SORT_ACTION_TYPE, binding.LOOP_GRAPH),
            (wl.SORT_DATA, binding.LOOP_ASYNC), (wl.SORT_NONE, binding.LOOP_PERSISTENT))
    with binding.Context(prob) as ctx:
        ctx.set_async_warps(True)
        for (policy, mode), b in zip(runs, batches):
            ctx.set_sort_policy(policy)
            ctx.add_events(b)
            ctx.run_events(mode)
        n = len(batches[0])
        hist, _ = ctx.read_history(0, 4 * n)
    for k, b in enumerate(batches):
        o = run_oracle(prob, b)
        np.testing.assert_array_equal(hist["steps"][k * n:(k + 1) * n], o["hist"]["steps"])
        np.testing.assert_array_equal(hist["secondaries"][k * n:(k + 1) * n], o["hist"]["secondaries"])


@pytest.mark.parametrize("warps", [False, True])
def test_parent_slot_reuse_keeps_histories(warps):
    prob = wl.water_cube_problem(history_capacity=2000, sort_policy=wl.SORT_LOCAL)
    prim = wl.water_cube_primaries()
    with binding.Context(prob) as ctx:
        ctx.set_async_warps(warps)
        ctx.set_parent_reuse(True)
        ctx.add_events(prim)
        ctx.run_events(binding.LOOP_ASYNC)
        hist, edep = ctx.read_history(0, len(prim))
    o = run_oracle(prob, prim)
    np.testing.assert_array_equal(hist["steps"], o["hist"]["steps"])
    np.testing.assert_array_equal(hist["secondaries"], o["hist"]["secondaries"])
    np.testing.assert_allclose(edep, o["edep"], rtol=1e-9, atol=1e-9 * 10.0)


@pytest.mark.parametrize("warps", [False, True])
def test_event_results_same_alone_and_mixed(warps):
    events = [e[:80] for e in wl.offload_events(6)]
    prob = wl.calorimeter_problem(1 << 15, Bz=4.0, max_events=8, sort_policy=wl.SORT_LOCAL)
    mix = wl.concat_primaries(events)
    g_mix = run_async(prob, mix, wl.SORT_LOCAL, warps)
    for k, ev in enumerate(events):
        g1 = run_gpu(prob, ev, mode=binding.LOOP_PERSISTENT)
        sl = slice(sum(len(e) for e in events[:k]), sum(len(e) for e in events[: k + 1]))
        np.testing.assert_array_equal(g_mix["hist"]["steps"][sl], g1["hist"]["steps"])
        np.testing.assert_array_equal(g_mix["hist"]["secondaries"][sl], g1["hist"]["secondaries"])
        e_id = int(ev["event"][0])
        t_mix, esc_mix = g_mix["tally"][e_id]
        t_one, esc_one = g1["tally"][e_id]
        np.testing.assert_allclose(t_mix, t_one, rtol=1e-12, atol=1e-9)
        assert esc_mix == pytest.approx(esc_one, rel=1e-12, abs=1e-9)


def test_rejects_other_policies():
    prob = wl.water_cube_problem(sort_policy=wl.SORT_ACTION_TYPE)
    with binding.Context(prob) as ctx:
        ctx.add_events(wl.water_cube_primaries(10))
        with pytest.raises(binding.CelerError) as ei:
            ctx.run_events(binding.LOOP_ASYNC)
        assert ei.value.status == 1
        ctx.set_sort_policy(wl.SORT_LOCAL)
        ctx.run_events(binding.LOOP_ASYNC)
        assert ctx.stats()["alive"] == 0


@pytest.mark.parametrize("policy,warps", SCHEDULES, ids=SCHED_IDS)
def test_budgeted_runs_keep_histories(policy, warps):
    """Short budgeted asynchronous runs, one after the other, interleaved
    with synchronous iterations: each run leaves every track between two
    steps, so the histories are the oracle's."""
    prob = wl.water_cube_problem(n_slots=1024, history_capacity=2000, sort_policy=policy)
    prim = wl.water_cube_primaries()
    with binding.Context(prob) as ctx:
        ctx.set_async_warps(warps)
        ctx.add_events(prim)
        runs = 0
        while True:
            done = ctx.run_iterations(binding.LOOP_ASYNC, budget=3)
            assert done <= 3 or warps  # passes are exact; per-warp pieces end by draining
            if runs % 3 == 2:
                ctx.run_iterations(binding.LOOP_PERSISTENT, budget=2)
            runs += 1
            s = ctx.stats()
            if s["alive"] == 0 and s["queued"] == 0:
                break
            assert runs < 20000
        hist, edep = ctx.read_history(0, len(prim))
    assert runs > 3
    o = run_oracle(prob, prim)
    np.testing.assert_array_equal(hist["steps"], o["hist"]["steps"])
    np.testing.assert_array_equal(hist["secondaries"], o["hist"]["secondaries"])
    np.testing.assert_allclose(edep, o["edep"], rtol=1e-9, atol=1e-9 * 10.0)


@pytest.mark.parametrize("warps", [False, True])
def test_stuck_run_ends_with_capacity_status(warps):
    """One slot and a one-entry buffer: the electron's second secondary can
    never be placed and no block can read the queued entry. No track steps
    any more, so after about a second every block leaves its loop and the
    host reads CELER_ERR_CAPACITY; the context stays usable."""
    prob = wl.calorimeter_problem(1, init_capacity=1, history_capacity=1, sort_policy=wl.SORT_LOCAL)
    prim = wl.electron_beam(1, 1000.0)
    with binding.Context(prob, max_iterations=10**9) as ctx:
        ctx.set_async_warps(warps)
        ctx.add_events(prim)
        with pytest.raises(binding.CelerError) as ei:
            ctx.run_events(binding.LOOP_ASYNC)
        assert ei.value.status == 2
        s = ctx.stats()
        assert s["alive"] == 1 and s["queued"] == 1


def test_warp_scheduling_switch_is_validated():
    prob = wl.water_cube_problem(sort_policy=wl.SORT_LOCAL)
    with binding.Context(prob) as ctx:
        lib = binding.load()
        assert lib.celer_set_async_warps(ctx._h, 2) == 1
        assert lib.celer_set_async_warps(ctx._h, -1) == 1
        assert lib.celer_set_async_warps(ctx._h, 1) == 0


def test_blocks_over_the_warp_queue_capacity_fall_back_to_passes():
    """Per-warp scheduling holds at most 1024 live tracks per block: two
    blocks that start the run with ~1500 each (left by one synchronous
    iteration) run block passes instead, with the oracle's histories."""
    prob = wl.water_cube_problem(n_slots=16384, history_capacity=8000, sort_policy=wl.SORT_LOCAL)
    prim = wl.water_cube_primaries(8000)
    with binding.Context(prob) as ctx:
        ctx.set_grid_blocks(2)
        ctx.add_events(prim)
        ctx.run_iterations(binding.LOOP_PERSISTENT, budget=1)
        state = ctx.debug_slots()
        live = state["status"] != 0
        owner = (np.arange(len(live)) // 32) % 2
        assert min(live[owner == 0].sum(), live[owner == 1].sum()) > 1024
        ctx.set_async_warps(True)
        ctx.run_events(binding.LOOP_ASYNC)
        hist, edep = ctx.read_history(0, len(prim))
    o = run_oracle(prob, prim)
    np.testing.assert_array_equal(hist["steps"], o["hist"]["steps"])
    np.testing.assert_array_equal(hist["secondaries"], o["hist"]["secondaries"])
    np.testing.assert_allclose(edep, o["edep"], rtol=1e-9, atol=1e-9 * 10.0)


def test_blocks_owning_more_than_16_bit_slot_indices_fall_back_to_passes():
    """One block owning 70,000 slots: its queue entries could not hold the
    slot indices, so it runs block passes."""
    prob = wl.water_cube_problem(n_slots=70000, history_capacity=500, sort_policy=wl.SORT_LOCAL)
    prim = wl.water_cube_primaries(500)
    with binding.Context(prob) as ctx:
        ctx.set_grid_blocks(1)
        ctx.set_async_warps(True)
        ctx.add_events(prim)
        ctx.run_events(binding.LOOP_ASYNC)
        hist, edep = ctx.read_history(0, len(prim))
    o = run_oracle(prob, prim)
    np.testing.assert_array_equal(hist["steps"], o["hist"]["steps"])
    np.testing.assert_allclose(edep, o["edep"], rtol=1e-9, atol=1e-9 * 10.0)
