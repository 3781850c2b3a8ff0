"""Shared helpers of the GPU parity tests: run a workload through the C ABI
and through the CPU oracle on the same seeded inputs."""
import os

import numpy as np

import oracle
from paper_2503_17608_gb300 import binding, workloads as wl


def run_gpu(prob, prim, mode=binding.LOOP_PERSISTENT, history=True, policy=None, stream=None, split=None):
    if policy is not None:
        prob = prob.replace(sort_policy=policy)
    if split is not None:
        prob = prob.replace(split_actions=int(split))
    if history:
        prob = prob.replace(history_capacity=len(prim))
    with binding.Context(prob, stream=stream) as ctx:
        ctx.add_events(prim)
        ctx.run_events(mode)
        stats = ctx.stats()
        out = dict(stats=stats)
        if history:
            out["hist"], out["edep"] = ctx.read_history(0, len(prim))
        events = list(dict.fromkeys(prim["event"].tolist()))
        out["tally"] = {}
        for e in events:
            out["tally"][e] = ctx.read_tallies(e)
    return out


def run_oracle(prob, prim, threads=None):
    hist, edep = oracle.World(prob).run(prim, n_threads=threads)
    return dict(hist=hist, edep=edep)


def match_fraction(g, o, rtol=1e-9, label=None):
    """Fraction of primaries whose integer counts are equal and deposits agree
    (each history's bins relative to its largest bin); the observed fraction
    is printed with the test's name."""
    same_int = (g["hist"]["steps"] == o["hist"]["steps"]) & (g["hist"]["secondaries"] == o["hist"]["secondaries"])
    scale = np.maximum(np.abs(o["edep"]).max(axis=1, keepdims=True), 1e-300)
    close = np.all(np.abs(g["edep"] - o["edep"]) <= rtol * scale, axis=1)
    mask = same_int & close
    frac = float(np.mean(mask)) if len(mask) else 1.0
    report(label or os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0], frac, len(mask))
    return frac, mask


def assert_conservation(prim, tally_by_event, rel=1e-12):
    for e, (tally, escaped) in tally_by_event.items():
        E0 = prim["E"][prim["event"] == e].sum()
        assert abs(tally.sum() + escaped - E0) <= rel * E0, (e, tally.sum() + escaped, E0)


def report(label, frac, n):
    """Print an observed match fraction (pytest -s shows it); the thresholds in
    the tests sit just below the fractions these lines recorded."""
    print(f"PARITY {label}: {frac:.4f} of {n} histories match the oracle", flush=True)


def assert_history_conservation(prim, hist, rel=1e-12):
    """Every history, matching the oracle or not, conserves its energy:
    deposited + escaped = the primary's energy."""
    np.testing.assert_allclose(hist["edep"] + hist["escaped"], prim["E"], rtol=rel)


def assert_event_tallies(prim, tally_by_event, g_edep, o_edep, mask, rtol=1e-9):
    """Each event's tally equals the oracle's histories where they match and the
    GPU's own history records where a last-bit branch flip made them differ
    (tally bins relative to the event's largest bin)."""
    for e, (tally, _) in tally_by_event.items():
        sel = prim["event"] == e
        want = np.where(mask[sel, None], o_edep[sel], g_edep[sel]).sum(0)
        scale = max(np.abs(want).max(), 1e-300)
        np.testing.assert_allclose(tally, want, rtol=0, atol=rtol * scale)
