"""Continuous batching (serving) and the autotuner, through the C ABI.

An event's results must not depend on which other events share the slot
store with it: its random streams depend only on (seed, event, track id,
draw index), so integer counts are identical and deposits differ only by the
order of floating-point atomic additions (1e-12 relative)."""
import numpy as np
import pytest

from paper_2503_17608_gb300 import binding, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    binding.load()


def small_events(n_events=12, cap=60):
    return [e[:cap] for e in wl.offload_events(n_events)]


@pytest.mark.parametrize("mode,policy", [(binding.LOOP_PERSISTENT, wl.SORT_ACTION_TYPE),
                                         (binding.LOOP_GRAPH, wl.SORT_ACTION_TYPE),
                                         (binding.LOOP_ASYNC, wl.SORT_LOCAL), (binding.LOOP_ASYNC, wl.SORT_DATA)])
def test_served_events_match_alone(mode, policy):
    """Chunks of the asynchronous loop end by draining (per-warp schedule)
    or after whole passes, so events admitted between chunks see the same
    histories as in the synchronous loops."""
    events = small_events()
    prob = wl.calorimeter_problem(1 << 14, Bz=4.0, max_events=64, sort_policy=policy)
    # arrivals close together so that events overlap on the device
    reqs = [(0.002 * i, int(e["event"][0]), e) for i, e in enumerate(events)]
    with binding.Context(prob) as ctx:
        res, summ, tallies = ctx.serve(reqs, mode=mode, chunk_iterations=4, with_tallies=True)
    assert summ["completed"] == len(events) and summ["admitted"] == len(events)
    assert np.all(res["done_s"] >= res["admit_s"]) and np.all(res["admit_s"] >= res["arrival_s"] - 1e-9)
    for k, e in enumerate(events):
        assert res["edep"][k] + res["escaped"][k] == pytest.approx(e["E"].sum(), rel=1e-12)
        with binding.Context(prob) as ctx:
            ctx.add_events(e)
            ctx.run_events(mode)
            t1, esc1 = ctx.read_tallies(int(e["event"][0]))
        np.testing.assert_allclose(tallies[k], t1, rtol=1e-12, atol=1e-9)
        assert res["escaped"][k] == pytest.approx(esc1, rel=1e-12, abs=1e-9)


def test_one_event_at_a_time_serving():
    events = small_events(6)
    prob = wl.calorimeter_problem(1 << 14, Bz=4.0, max_events=8)
    reqs = [(0.0, int(e["event"][0]), e) for e in events]
    with binding.Context(prob) as ctx:
        res, summ, _ = ctx.serve(reqs, max_in_flight=1)
    order = np.argsort(res["admit_s"])
    # each event is admitted only after the previous one finished
    assert np.all(res["admit_s"][order][1:] >= res["done_s"][order][:-1])
    assert summ["completed"] == len(events)


def test_serving_reuses_tally_rows():
    events = small_events(10, cap=20)
    prob = wl.calorimeter_problem(1 << 13, max_events=3)
    reqs = [(0.0005 * i, 100 + i, e) for i, e in enumerate(events)]
    for i, e in enumerate(events):
        e["event"][:] = 100 + i
    with binding.Context(prob) as ctx:
        res, summ, _ = ctx.serve(reqs)
    assert summ["completed"] == len(events)
    for k, e in enumerate(events):
        assert res["edep"][k] + res["escaped"][k] == pytest.approx(e["E"].sum(), rel=1e-12)


def test_autotuner_picks_a_measured_best():
    events = small_events(8, cap=40)
    prim = wl.concat_primaries(events)
    prob = wl.calorimeter_problem(1 << 12, Bz=4.0, max_events=16)
    best, trials = binding.autotune(prob, prim, [1 << 12, 1 << 13], [128, 256], [wl.SORT_NONE, wl.SORT_ACTION_TYPE],
                                    [binding.LOOP_PERSISTENT])
    assert len(trials) == 8
    assert all(t["track_steps_per_s"] > 0 for t in trials)
    assert best["track_steps_per_s"] == max(t["track_steps_per_s"] for t in trials)


def test_autotuner_tries_both_schedules_of_the_asynchronous_loop():
    events = small_events(8, cap=40)
    prim = wl.concat_primaries(events)
    prob = wl.calorimeter_problem(1 << 12, Bz=4.0, max_events=16)
    best, trials = binding.autotune(prob, prim, [1 << 12], [256], [wl.SORT_LOCAL, wl.SORT_DATA, wl.SORT_NONE],
                                    [binding.LOOP_ASYNC, binding.LOOP_PERSISTENT])
    combos = sorted((t["sort_policy"], t["mode"], t["async_warps"]) for t in trials)
    A, P = binding.LOOP_ASYNC, binding.LOOP_PERSISTENT
    assert combos == sorted([(wl.SORT_LOCAL, A, 1), (wl.SORT_LOCAL, A, 0), (wl.SORT_LOCAL, P, 1),
                             (wl.SORT_DATA, A, 1), (wl.SORT_DATA, P, 1), (wl.SORT_NONE, A, 1), (wl.SORT_NONE, P, 1)])
    for t in trials:
        runnable = not (t["mode"] == A and t["sort_policy"] == wl.SORT_NONE)
        assert (t["track_steps_per_s"] > 0) == runnable
    assert best["track_steps_per_s"] == max(t["track_steps_per_s"] for t in trials)


def test_consecutive_admissions_track_the_buffer_fill_level():
    """celer_add_primaries reads the buffer's fill level from the device only
    after step work; between two runs it counts its own pushes. A second
    batch that would overflow the buffer is refused without a run in between,
    and after a run the space is back."""
    prob = wl.calorimeter_problem(1 << 10, init_capacity=64, max_events=4)
    a = wl.electron_beam(40, 50.0, event=0)
    b = wl.electron_beam(30, 50.0, event=1)
    c = wl.electron_beam(20, 50.0, event=2)
    with binding.Context(prob) as ctx:
        ctx.add_primaries(0, a)
        with pytest.raises(binding.CelerError) as ei:
            ctx.add_primaries(1, b)  # 40 + 30 > 64
        assert ei.value.status == 2
        ctx.add_primaries(2, c)  # 40 + 20 fits
        assert ctx.stats()["queued"] == 60
        ctx.run_events(binding.LOOP_PERSISTENT)
        ctx.add_primaries(1, b)  # the buffer drained
        ctx.run_events(binding.LOOP_ASYNC if prob.sort_policy in (wl.SORT_LOCAL, wl.SORT_DATA)
                       else binding.LOOP_PERSISTENT)
        for e, ev in ((0, a), (1, b), (2, c)):
            tally, esc = ctx.read_tallies(e)
            assert tally.sum() + esc == pytest.approx(ev["E"].sum(), rel=1e-12)
