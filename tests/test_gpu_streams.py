"""Event-per-stream mode (paper Sec. 4.1) and per-iteration hit readout
(Sec. 3.4): contexts on their own streams, each with part of the GPU's
blocks, stepping events side by side from host threads, give every event the
tallies it gets alone; the hit buffer holds the tallies after each run."""
import threading

import numpy as np
import pytest

from paper_2503_17608_gb300 import binding, workloads as wl

pytestmark = pytest.mark.gpu


def events(n, per_event=6):
    prob, _ = wl.calorimeter_1gev(1)
    evs = []
    for e in range(n):
        p = wl.electron_beam(per_event, 200.0 + 50.0 * e, event=e)
        evs.append(p)
    return prob.replace(n_slots=4096, max_events=1, sort_policy=wl.SORT_LOCAL), evs


def alone(prob, evs):
    out = []
    with binding.Context(prob) as ctx:
        for e, ev in enumerate(evs):
            ctx.reset_event(e)
            ctx.add_primaries(e, ev)
            ctx.run_events(binding.LOOP_PERSISTENT)
            out.append(ctx.read_tallies(e))
    return out


@pytest.mark.parametrize("hit_mode", [1, 2])
def test_event_per_stream_matches_alone(hit_mode):
    import torch

    prob, evs = events(8)
    ref = alone(prob, evs)
    k_streams = 2
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    streams = [torch.cuda.Stream() for _ in range(k_streams)]
    ctxs = [binding.Context(prob, stream=s.cuda_stream) for s in streams]
    hits = []
    for c in ctxs:
        c.set_grid_blocks(sms // k_streams)
        h = torch.zeros(c.n_bins, dtype=torch.float64, pin_memory=True)
        c.set_hit_readout(hit_mode, h)
        hits.append(h)
    got = [None] * len(evs)
    last_hits = [None] * len(evs)
    errors = []

    def worker(k):
        try:
            c = ctxs[k]
            for e in range(k, len(evs), k_streams):
                c.reset_event(e)
                c.add_primaries(e, evs[e])
                c.run_events(binding.LOOP_HOST)
                got[e] = c.read_tallies(e)
                last_hits[e] = hits[k].numpy().copy()
        except Exception as exc:
            errors.append(exc)

    th = [threading.Thread(target=worker, args=(k,)) for k in range(k_streams)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for c in ctxs:
        c.close()
    assert not errors, errors
    for e in range(len(evs)):
        np.testing.assert_allclose(got[e][0], ref[e][0], rtol=1e-12, atol=1e-9)
        assert got[e][1] == pytest.approx(ref[e][1], rel=1e-12, abs=1e-9)
        # the copy after the last iteration holds the event's final tallies
        np.testing.assert_allclose(last_hits[e], got[e][0], rtol=0, atol=0)


def test_hit_readout_and_grid_arguments():
    import torch

    prob, evs = events(1)
    with binding.Context(prob) as ctx:
        short = torch.zeros(ctx.n_bins - 1, dtype=torch.float64, pin_memory=True)
        with pytest.raises(binding.CelerError):
            ctx.set_hit_readout(1, short)
        with pytest.raises(binding.CelerError):
            ctx.set_hit_readout(3, torch.zeros(ctx.n_bins, dtype=torch.float64, pin_memory=True))
        with pytest.raises(binding.CelerError):
            ctx.set_grid_blocks(-1)
        ctx.set_grid_blocks(1)  # one block: still correct, only slower
        for mode in (binding.LOOP_HOST, binding.LOOP_GRAPH, binding.LOOP_PERSISTENT):
            ctx.reset_event(0)
            ctx.add_primaries(0, evs[0])
            ctx.run_events(mode)
            tally, esc = ctx.read_tallies(0)
            assert tally.sum() + esc == pytest.approx(evs[0]["E"].sum(), rel=1e-12)
