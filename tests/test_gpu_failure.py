"""Failure detection without a GPU fault: the persistent loops' grid-barrier
wait is bounded. A block that never arrives makes the others give up after a
short cycle limit, raise the abort word and the timeout error bit, and end,
and the device stays usable (no trap, no hang)."""
import numpy as np
import pytest

from paper_2503_17608_gb300 import binding, workloads as wl

pytestmark = pytest.mark.gpu

ERR_BARRIER_TIMEOUT = 32
CELER_OK, CELER_ERR_TIMEOUT = 0, 4


def test_barrier_passes_when_every_block_arrives():
    st, err, ab = binding.debug_barrier_timeout(4, -1, 2_000_000)
    assert st == CELER_OK and err == 0 and ab == 0


@pytest.mark.parametrize("absent", [0, 3])
def test_barrier_gives_up_when_a_block_never_arrives(absent):
    st, err, ab = binding.debug_barrier_timeout(4, absent, 2_000_000)  # ~1 ms at 2 GHz
    assert st == CELER_ERR_TIMEOUT
    assert err & ERR_BARRIER_TIMEOUT
    assert ab == 1
    # the device is still usable: a transport run afterwards is correct
    prob = wl.water_cube_problem(n_slots=1024)
    prim = wl.water_cube_primaries(100)
    with binding.Context(prob) as ctx:
        ctx.add_events(prim)
        ctx.run_events(binding.LOOP_PERSISTENT)
        tally, esc = ctx.read_tallies(0)
    assert tally.sum() + esc == pytest.approx(prim["E"].sum(), rel=1e-12)


def test_barrier_probe_rejects_bad_arguments():
    for args in [(1, 0, 1000), (9, 0, 1000), (4, 4, 1000), (4, -2, 1000), (4, 0, 0)]:
        st, _, _ = binding.debug_barrier_timeout(*args)
        assert st == 1  # CELER_ERR_INVALID


@pytest.mark.parametrize("which", [0, 1], ids=["buffer-entry", "warp-queue-entry"])
def test_queue_wait_gives_up_when_nothing_writes_the_entry(which):
    """The asynchronous loop's waits for a buffer entry or a shared-memory
    queue entry are bounded the same way: nothing writes the entry, the wait
    gives up, raises the abort word and the timeout bit, and the device stays
    usable for a run of the asynchronous loop."""
    st, err, ab = binding.debug_queue_wait(which, 2_000_000)
    assert st == CELER_ERR_TIMEOUT
    assert err & ERR_BARRIER_TIMEOUT
    assert ab == 1
    prob = wl.water_cube_problem(n_slots=1024, sort_policy=wl.SORT_LOCAL)
    prim = wl.water_cube_primaries(100)
    with binding.Context(prob) as ctx:
        ctx.add_events(prim)
        ctx.run_events(binding.LOOP_ASYNC)
        tally, esc = ctx.read_tallies(0)
    assert tally.sum() + esc == pytest.approx(prim["E"].sum(), rel=1e-12)


@pytest.mark.parametrize("which", [2, 3])
def test_queue_wait_passes_when_the_entry_is_written(which):
    st, err, ab = binding.debug_queue_wait(which, 2_000_000)
    assert st == CELER_OK and err == 0 and ab == 0


def test_queue_wait_probe_rejects_bad_arguments():
    for args in [(-1, 1000), (4, 1000), (0, 0), (1, 5_000_000_000)]:
        st, _, _ = binding.debug_queue_wait(*args)
        assert st == 1  # CELER_ERR_INVALID
