"""The step kernels' rejection samplers decide each attempt in FP32 and fall
back to FP64 near the acceptance boundary. These tests check, on millions of
records spanning the workloads' energies and the filter's edges, that they
give bit-identical samples, draw counts and flags to the plain FP64 samplers
(the form the parity tests against the CPU oracle were established with)."""
import numpy as np
import pytest

from paper_2503_17608_gb300 import binding

pytestmark = pytest.mark.gpu

ME = 0.51099895


def records(rng, n, lo, hi, extra=()):
    E = np.concatenate([np.exp(rng.uniform(np.log(lo), np.log(hi), n)), np.asarray(extra, np.float64)])
    tid = rng.integers(0, 2**63, len(E), dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, len(E), dtype=np.uint64)
    ctr = rng.integers(0, 1000, len(E)).astype(np.uint32)
    return E, tid, ctr


def assert_same(a, b):
    for x, y, name in zip(a, b, ("eps", "cost", "ctr", "ok")):
        assert np.array_equal(x, y), f"{name} differs in {np.count_nonzero(x != y)} of {len(x)} records"


def test_compton_filtered_equals_fp64():
    rng = np.random.default_rng(11)
    # photon energies of the workloads (0.01 MeV .. 10 GeV), plus the edges of
    # the filter's range k = E/m in [1e-4, 1e6] and outside it
    edges = [ME * 1e-4, ME * 1e-4 * (1 + 1e-15), ME * 0.99e-4, ME * 1e6, ME * 1.01e6, 1.022, 0.511, 1e4]
    E, tid, ctr = records(rng, 3_000_000, 0.01, 1e4, edges)
    filt = binding.debug_sample(0, E, tid, ctr)
    ref = binding.debug_sample(1, E, tid, ctr)
    assert_same(filt, ref)
    eps, cost, c, ok = filt
    assert ok.all()
    assert (c > ctr).all() and ((c - ctr) % 3 == 0).all()
    eps0 = 1.0 / (1.0 + 2.0 * E / ME)
    assert ((eps >= eps0 * (1 - 1e-15)) & (eps <= 1.0)).all()
    assert ((cost >= -1.0 - 1e-12) & (cost <= 1.0)).all()


def test_compton_low_energy_forward_region():
    # small k: eps near 1, where 1 - eps and 2b - a are small (the filter's
    # cancellation-free forms and its tiny-value fallback)
    rng = np.random.default_rng(12)
    E, tid, ctr = records(rng, 1_000_000, ME * 1e-4, 0.02)
    assert_same(binding.debug_sample(0, E, tid, ctr), binding.debug_sample(1, E, tid, ctr))


def test_moller_filtered_equals_fp64():
    rng = np.random.default_rng(13)
    cut = 1.0
    E, tid, ctr = records(rng, 3_000_000, 2.0 * cut * (1 + 1e-12), 1e4, [2.0000001, 2.5, 1e4, 3e8])
    filt = binding.debug_sample(2, E, tid, ctr, cut=cut)
    ref = binding.debug_sample(3, E, tid, ctr, cut=cut)
    assert_same(filt, ref)
    eps, _, c, ok = filt
    assert ok.all()
    assert (c > ctr).all() and ((c - ctr) % 2 == 0).all()
    x = cut / E
    assert ((eps >= x * (1 - 1e-15)) & (eps <= 0.5 * (1 + 1e-15))).all()


def test_moller_other_cuts():
    rng = np.random.default_rng(14)
    for cut in (0.01, 0.1, 10.0):
        E, tid, ctr = records(rng, 300_000, 2.0 * cut * 1.000001, 1e4)
        assert_same(binding.debug_sample(2, E, tid, ctr, cut=cut), binding.debug_sample(3, E, tid, ctr, cut=cut))
