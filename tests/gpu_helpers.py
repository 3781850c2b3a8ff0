"""Shared helpers of the GPU parity tests: run a workload through the C ABI
and through the CPU oracle on the same seeded inputs."""
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


def match_fraction(g, o, rtol=1e-9):
    """Fraction of primaries whose integer counts are equal and deposits agree."""
    same_int = (g["hist"]["steps"] == o["hist"]["steps"]) & (g["hist"]["secondaries"] == o["hist"]["secondaries"])
    scale = np.maximum(np.abs(o["edep"]).max(axis=1, keepdims=True), 1e-300)
    close = np.all(np.abs(g["edep"] - o["edep"]) <= rtol * scale, axis=1)
    return float(np.mean(same_int & close)), same_int & close


def assert_conservation(prim, tally_by_event, rel=1e-12):
    for e, (tally, escaped) in tally_by_event.items():
        E0 = prim["E"][prim["event"] == e].sum()
        assert abs(tally.sum() + escaped - E0) <= rel * E0, (e, tally.sum() + escaped, E0)
