"""Table-driven log/exp and sin/cos of the step kernels (Tang's method)
against CUDA's own routines and numpy's, in units in the last place."""
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
    for fn in (-1, 12):
        with pytest.raises(Exception):
            binding.debug_math(fn, np.ones(3))


def test_fast_sincos_2pi_absolute_error():
    rng = np.random.default_rng(8)
    u = np.concatenate([rng.uniform(0, 1, 400000), rng.uniform(0, 1e-6, 20000), 1.0 - rng.uniform(0, 1e-6, 20000),
                        np.array([0.0, 0.25, 0.5, 0.75, 1.0, 2.0 ** -53, 1.0 - 2.0 ** -53])])
    s = binding.debug_math(4, u)
    c = binding.debug_math(5, u)
    # reference in extended precision (2 pi u rounded in binary64 alone is
    # off by up to 4.4e-16 near u = 1)
    twopi = 2 * np.longdouble("3.141592653589793238462643383279502884")
    ul = u.astype(np.longdouble)
    ref_s = np.sin(twopi * ul)
    ref_c = np.cos(twopi * ul)
    assert float(np.max(np.abs(s - ref_s))) < 2.5e-16
    assert float(np.max(np.abs(c - ref_c))) < 2.5e-16
    # CUDA's sin(2 pi u) carries the rounding of 2 pi u
    assert np.max(np.abs(s - binding.debug_math(6, u))) < 8e-16
    assert np.max(np.abs(c - binding.debug_math(7, u))) < 8e-16
    assert np.max(np.abs(s * s + c * c - 1.0)) < 4.5e-16


def test_fast_sincos_outside_unit_interval_follows_library():
    u = np.array([-0.25, 1.25, 3.5, -2.0])
    np.testing.assert_allclose(binding.debug_math(4, u), np.sin(2 * np.pi * u), atol=1e-15)
    np.testing.assert_allclose(binding.debug_math(5, u), np.cos(2 * np.pi * u), atol=1e-15)


def test_fast_sincos_of_turn_angles_within_two_ulp():
    """sin and cos of a helix half-turn (any angle up to ~1e5 rad, Cody-Waite
    reduction onto the 256-entry table) against CUDA's and numpy's."""
    rng = np.random.default_rng(8)
    x = np.concatenate([rng.uniform(-50, 50, 300000), rng.uniform(-1e4, 1e4, 100000),
                        rng.uniform(-1e-3, 1e-3, 100000), np.exp(rng.uniform(-30, 11, 100000)),
                        np.array([0.0, 1e-300, np.pi, -np.pi, np.pi / 2, 1e5 * 0.999])])
    for fast_fn, cuda_fn, ref in ((8, 10, np.sin), (9, 11, np.cos)):
        fast = binding.debug_math(fast_fn, x)
        cuda = binding.debug_math(cuda_fn, x)
        exact = ref(x)
        # ulps of the result, or absolute 2.5e-16 near zeros of sin / cos
        ok_c = (ulps(fast, cuda) <= 2.0) | (np.abs(fast - cuda) <= 2.5e-16)
        ok_r = (ulps(fast, exact) <= 2.0) | (np.abs(fast - exact) <= 2.5e-16)
        assert ok_c.all(), x[~ok_c][:5]
        assert ok_r.all(), x[~ok_r][:5]


def test_fast_sincos_outside_range_follows_cuda():
    x = np.array([1e5, -2e5, 1e300, np.inf, np.nan])
    for fast_fn, cuda_fn in ((8, 10), (9, 11)):
        fast = binding.debug_math(fast_fn, x)
        cuda = binding.debug_math(cuda_fn, x)
        np.testing.assert_array_equal(np.isnan(fast), np.isnan(cuda))
        ok = ~np.isnan(cuda)
        np.testing.assert_array_equal(fast[ok], cuda[ok])


def test_fp64_rate_probe():
    """The FP64 throughput probe behind the bench's ALU roofline: at most the
    derived peak (2 FP64 FMA per SM-cycle at the maximum clock), and well
    above a fraction of it; bad arguments are refused."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    derived = 2 * 2 * sms * 2.07e9 / 1e12
    tflops, ms = binding.debug_fp64_rate(4, 20000)
    assert ms > 0.0
    assert 0.3 * derived < tflops <= 1.05 * derived, (tflops, derived)
    for bad in ((0, 100), (9, 100), (4, 0)):
        with pytest.raises(binding.CelerError) as ei:
            binding.debug_fp64_rate(*bad)
        assert ei.value.status == 1


def test_lane_counters_are_absent_from_the_product_build():
    """The active-lane counters exist only in the diagnostic build; the
    product library answers CELER_ERR_STATE."""
    with pytest.raises(binding.CelerError) as ei:
        binding.debug_lane_counts()
    assert ei.value.status == 5
