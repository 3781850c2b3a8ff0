"""The two-sample layer-profile tests used between the CUDA path and the
oracle (independent seeds): they pass for two oracle runs that differ only in
their seed, and they reject plausible mistakes of the size that matters
(radiation length 10 % off, deposits 2 % too high, one layer off, two layers
swapped). CPU only: both samples come from the oracle."""
import dataclasses

import pytest

import oracle
from paper_2503_17608_gb300 import workloads as wl
from stats_helpers import layer_profile_tests

N = 10000


@pytest.fixture(scope="module")
def base():
    prob, prim = wl.calorimeter_1gev(N)
    _, e = oracle.World(prob.replace(seed=12)).run(prim)
    return prob, prim, e


@pytest.mark.parametrize("seed", [13, 14])
def test_independent_seeds_pass(base, seed):
    prob, prim, e12 = base
    _, e = oracle.World(prob.replace(seed=seed)).run(prim)
    p_layer, p_t2, k = layer_profile_tests(e12, e)
    assert k == prob.n_layers_total
    assert p_layer > 1e-3 and p_t2 > 1e-3, (p_layer, p_t2)


def test_radiation_length_off_by_ten_percent_is_rejected(base):
    prob, prim, e12 = base
    m = prob.materials
    wrong = type(m)([dataclasses.replace(m[0], X0=1.1 * m[0].X0)] + list(m[1:]))
    _, e = oracle.World(prob.replace(seed=13, materials=wrong)).run(prim)
    _, p_t2, _ = layer_profile_tests(e12, e)
    assert p_t2 < 1e-6


def test_deposit_scale_and_layer_mistakes_are_rejected(base):
    prob, prim, e12 = base
    _, e = oracle.World(prob.replace(seed=13)).run(prim)
    assert layer_profile_tests(e12, 1.02 * e)[1] < 1e-6
    shifted = e.copy()
    shifted[:, 1:] = e[:, :-1]
    shifted[:, 0] = 0.0
    assert layer_profile_tests(e12, shifted)[1] < 1e-6
    swapped = e.copy()
    swapped[:, [10, 11]] = e[:, [11, 10]]
    assert layer_profile_tests(e12, swapped)[1] < 1e-6
