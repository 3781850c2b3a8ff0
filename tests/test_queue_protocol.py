"""Model check, on the CPU, of the concurrent-queue protocol of the
asynchronous loop (the initializer buffer and the per-warp shared-memory
queues use the same one).

Entry i of a buffer of capacity C (stored at i mod C) has a state word:
2 lap (free for its writer), 2 lap + 1 (written), 2 lap + 2 (read), with
lap = i // C. Writers reserve indices on the tail only while
tail + n <= head + C (head: the readers' claims), then wait for "free",
write and publish "written". Readers claim written entries on an
availability count (undone if short), take indices from the head, wait for
"written", read and publish "read". Tracks end at random; an ended track's
count goes to `finished` after its reservations, and a reader that sees
finished == tail (read in that order) concludes that nothing is live or
queued.

Actors are Python generators that yield at every shared-memory access; a
seeded random scheduler interleaves them. The checks: every reserved entry
is read exactly once with the value written to it, no wait outlasts the
scheduler's bound (no deadlock), tail - head never exceeds C, and a reader
never concludes the end while work is live or queued."""
import random

import pytest


class Shared:
    def __init__(self, capacity, n_initial):
        self.C = capacity
        self.state = [0] * capacity
        self.value = [None] * capacity
        self.head = 0
        self.tail = n_initial
        self.avail = n_initial
        self.finished = 0
        for i in range(n_initial):  # entries written before the run
            self.state[i % capacity] = 2 * (i // capacity) + 1
            self.value[i % capacity] = ("primary", i)
        self.reads = {}
        self.live = 0  # tracks in slots (the model's ground truth)
        self.errors = []


def writer_reserve(sh, n):
    """Reserve n entries on the tail by compare-and-swap against the head;
    yields between the reads and the swap. Returns the first index or None."""
    for _ in range(64):
        h = sh.head
        yield
        cur = sh.tail
        yield
        if cur + n > h + sh.C:
            return None
        if sh.tail == cur:  # the swap
            sh.tail = cur + n
            if sh.tail - sh.head > sh.C:
                sh.errors.append("tail passed head + capacity")
            return cur
        yield
    return None


def write_entry(sh, index, value, bound):
    slot, lap2 = index % sh.C, 2 * (index // sh.C)
    for _ in range(bound):
        if sh.state[slot] == lap2:
            break
        yield
    else:
        sh.errors.append(f"writer of {index} waited forever")
        return
    sh.value[slot] = value
    yield
    sh.state[slot] = lap2 + 1
    sh.avail += 1


def read_entry(sh, index, bound):
    slot, lap2 = index % sh.C, 2 * (index // sh.C)
    for _ in range(bound):
        if sh.state[slot] == lap2 + 1:
            break
        yield
    else:
        sh.errors.append(f"reader of {index} waited forever")
        return None
    v = sh.value[slot]
    yield
    sh.state[slot] = lap2 + 2
    if index in sh.reads:
        sh.errors.append(f"entry {index} read twice")
    sh.reads[index] = v
    return v


def block(sh, rng, seed_id, max_secondaries, bound, count_first=False):
    """One block: claims a few entries, steps its tracks (each ends or makes
    secondaries), counts its ended tracks after their reservations, and
    leaves when finished == tail. count_first plants a mistake: a parent's
    end is counted before its secondaries are reserved."""
    mine = []
    made = 0
    while True:
        # claim on the availability count, then indices on the head
        a = sh.avail
        yield
        want = min(a, rng.randint(1, 3)) if a > 0 else 0
        if want > 0:
            old = sh.avail
            sh.avail -= want
            yield
            if old >= want:
                first = sh.head
                sh.head += want
                yield
                for k in range(want):
                    v = yield from read_entry(sh, first + k, bound)
                    if v is not None:
                        mine.append(v)
                        sh.live += 1
            else:
                sh.avail += want
                yield
        if not mine:
            f = sh.finished
            yield
            t = sh.tail
            yield
            if f == t:
                if sh.live != 0 or sh.tail != sh.head or sh.avail != 0:
                    sh.errors.append("end concluded with work left")
                return
            continue
        # one step of every track: end it, or let it make secondaries
        ended = 0
        keep = []
        for tr in mine:
            r = rng.random()
            if r < 0.5 and made < max_secondaries:
                n = rng.randint(1, 2)
                if count_first:
                    sh.finished += 1
                    sh.live -= 1
                    yield
                first = yield from writer_reserve(sh, n)
                if first is None:
                    keep.append(tr)  # deferred: the same step is tried again later
                    continue
                made += n
                for k in range(n):
                    yield from write_entry(sh, first + k, ("secondary", seed_id, made, k), bound)
                if not count_first:
                    ended += 1  # the parent ends with this step
            elif r < 0.8:
                ended += 1
            else:
                keep.append(tr)
        mine = keep
        sh.live -= ended
        yield
        sh.finished += ended  # after the block's reservations


def run(seed, n_blocks, capacity, n_primaries, max_secondaries, bound=5000, count_first=False):
    rng = random.Random(seed)
    sh = Shared(capacity, n_primaries)
    actors = [block(sh, random.Random(seed * 1000 + b), b, max_secondaries, bound, count_first)
              for b in range(n_blocks)]
    alive = list(range(n_blocks))
    steps = 0
    while alive:
        i = rng.choice(alive)
        try:
            next(actors[i])
        except StopIteration:
            alive.remove(i)
        steps += 1
        assert steps < 5_000_000, "scheduler bound reached (livelock)"
    return sh


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("capacity", [4, 16, 64])
def test_every_entry_read_once_and_the_end_is_exact(seed, capacity):
    sh = run(seed, n_blocks=5, capacity=capacity, n_primaries=min(capacity, 6), max_secondaries=12)
    assert sh.errors == []
    assert sorted(sh.reads) == list(range(sh.tail))  # every reserved entry read exactly once
    assert sh.head == sh.tail and sh.avail == 0 and sh.live == 0
    assert sh.finished == sh.tail
    primaries = [v for v in sh.reads.values() if v[0] == "primary"]
    assert sorted(p[1] for p in primaries) == list(range(min(capacity, 6)))


def test_a_misplaced_count_is_caught():
    """The end check is sensitive: counting a parent's end before its
    secondaries are reserved lets some reader conclude the end while work is
    live or queued, or leaves reserved entries unread."""
    caught = 0
    for seed in range(30):
        sh = run(seed, n_blocks=5, capacity=16, n_primaries=6, max_secondaries=12, count_first=True)
        if sh.errors or sorted(sh.reads) != list(range(sh.tail)):
            caught += 1
    assert caught > 0
