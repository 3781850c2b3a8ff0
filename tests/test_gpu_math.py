"""Table-driven log/exp of the step kernels (Tang's method) against CUDA's
own routines and numpy's, in units in the last place."""
import numpy as np
import pytest

from paper_2503_17608_gb300 import binding

pytestmark = pytest.mark.gpu


def ulps(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = np.spacing(np.maximum(np.abs(a), np.abs(b)))
    return np.abs(a - b) / scale


def log_args(rng):
    return np.concatenate([
        np.exp(rng.uniform(-700, 700, 200000)),          # all exponents
        1.0 + rng.uniform(-0.02, 0.02, 200000),           # around 1 (cancellation)
        rng.uniform(1e-3, 1e4, 200000),                   # energies, MeV
        (np.arange(1, 200001) - 0.5) * 2.0 ** -18,       # uniform draws
        np.array([1.0, 2.0, 0.75, 1.5, np.nextafter(1.0, 0), np.nextafter(1.0, 2), 2.0 ** -1022, 1.7e308]),
    ])


def test_fast_log_within_two_ulp_of_cuda_and_numpy():
    x = log_args(np.random.default_rng(5))
    fast = binding.debug_math(0, x)
    cuda = binding.debug_math(2, x)
    ref = np.log(x)
    assert ulps(fast, cuda).max() <= 2.0
    assert ulps(fast, ref).max() <= 2.0
    assert fast[np.where(x == 1.0)[0]].tolist() == [0.0]


def test_fast_log_special_arguments_follow_cuda():
    x = np.array([0.0, -1.0, np.inf, np.nan, 5e-324, 1e-310, -0.0])
    fast = binding.debug_math(0, x)
    cuda = binding.debug_math(2, x)
    np.testing.assert_array_equal(np.isnan(fast), np.isnan(cuda))
    ok = ~np.isnan(cuda)
    np.testing.assert_array_equal(fast[ok], cuda[ok])


def test_fast_exp_within_two_ulp_of_cuda_and_numpy():
    rng = np.random.default_rng(6)
    x = np.concatenate([rng.uniform(-707, 707, 300000), rng.uniform(-1, 1, 300000),
                        rng.uniform(-1e-6, 1e-6, 100000), np.array([0.0, 1.0, -1.0, 700.0, -700.0])])
    fast = binding.debug_math(1, x)
    cuda = binding.debug_math(3, x)
    assert ulps(fast, cuda).max() <= 2.0
    assert ulps(fast, np.exp(x)).max() <= 2.0
    assert fast[np.where(x == 0.0)[0]].tolist() == [1.0]


def test_fast_exp_outside_reduced_range_follows_cuda():
    x = np.array([708.0, 709.7, 710.0, -708.0, -745.0, -800.0, np.inf, -np.inf, np.nan])
    fast = binding.debug_math(1, x)
    cuda = binding.debug_math(3, x)
    np.testing.assert_array_equal(np.isnan(fast), np.isnan(cuda))
    ok = ~np.isnan(cuda)
    np.testing.assert_array_equal(fast[ok], cuda[ok])


def test_fast_log_exp_round_trip():
    x = np.random.default_rng(7).uniform(1e-3, 1e4, 100000)
    back = binding.debug_math(1, binding.debug_math(0, x))
    assert np.max(np.abs(back / x - 1.0)) < 1e-13


def test_invalid_function_code_is_rejected():
    with pytest.raises(Exception):
        binding.debug_math(4, np.ones(3))
