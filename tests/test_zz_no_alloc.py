"""The allocation-free partition entry point gives the same partition as the
step loop (checked through the existing diagnostics entry point), on two
calls in a row. Some callers cannot allocate device memory themselves (their
framework's caching allocator owns it, or they cannot pay for the device-wide
synchronisation of cudaFree); this call only uses a fixed array inside the
library. Collected last on purpose, and independent of the other tests."""
import numpy as np
import pytest

from paper_2503_17608_gb300 import binding, workloads as wl

pytestmark = pytest.mark.gpu


def test_noalloc_partition_matches_step_loop_partition():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    prob = wl.calorimeter_problem(4096, sort_policy=wl.SORT_ACTION_TYPE)
    prim = wl.electron_beam(12, 1000.0)
    compared = 0
    with binding.Context(prob) as ctx:
        ctx.add_events(prim)
        for it in range(40):
            ctx.step()
            if it not in (14, 15):  # two iterations, so two calls in a row
                continue
            keys, perm, offs = ctx.debug_partition()
            n_keys = len(offs) - 1
            d_keys = torch.from_numpy(keys.copy()).cuda()
            d_perm = torch.full((len(keys),), -1, dtype=torch.int32, device="cuda")
            d_offs = torch.zeros(n_keys + 1, dtype=torch.int32, device="cuda")
            binding.partition_keys_noalloc(d_keys.data_ptr(), len(keys), n_keys, n_keys - 1, d_perm.data_ptr(),
                                           d_offs.data_ptr(), torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            got_perm = d_perm.cpu().numpy().view(np.uint32)
            got_offs = d_offs.cpu().numpy().view(np.uint32)
            placed = offs[n_keys - 1]  # every slot but the vacant ones
            assert placed > 0
            np.testing.assert_array_equal(got_offs, offs)
            np.testing.assert_array_equal(got_perm[:placed], perm[:placed])
            compared += 1
    assert compared == 2


def test_noalloc_partition_rejects_oversized_input():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with pytest.raises(binding.CelerError) as ei:
        binding.partition_keys_noalloc(1, (1 << 20) + 1, 4, -1, 1, 1)
    assert ei.value.status == 1
    with pytest.raises(binding.CelerError):
        binding.partition_keys_noalloc(1, 100, 17, -1, 1, 1)


def _expected(keys, n_keys):
    """Stable partition by numpy: offsets from bincount of the in-range keys,
    and each key's slots in ascending order."""
    in_range = keys < n_keys
    counts = np.bincount(keys[in_range], minlength=n_keys)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint32)
    order = np.argsort(keys, kind="stable").astype(np.uint32)
    return offsets, order[: offsets[-1]]


@pytest.mark.parametrize("n", [1, 255, 257, 100003, 1 << 20])
def test_noalloc_partition_random_keys_against_numpy(n):
    """Random 8-bit keys, some of them out of range, n_keys from 1 to 16 and
    skip_key in the middle: the offsets equal numpy's bincount prefix, every
    placed slot equals numpy's stable argsort, and the positions that the call
    must not write (skip_key's range, and everything past the in-range slots)
    keep their old contents. n = 2^20 with 16 keys runs the single-block scan
    over its largest count array (16 x 4096 entries)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(n)
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(16, -1), (16, 15), (16, 7), (5, 2), (1, -1), (1, 0), (11, 10)]
    for n_keys, skip in cases:
        keys = rng.integers(0, n_keys + 3, size=n, dtype=np.uint8)  # ~3/(n_keys+3) out of range
        want_offs, want_perm = _expected(keys, n_keys)
        d_keys = torch.from_numpy(keys).cuda()
        d_perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        d_offs = torch.full((n_keys + 1,), -1, dtype=torch.int32, device="cuda")
        binding.partition_keys_noalloc(d_keys.data_ptr(), n, n_keys, skip, d_perm.data_ptr(), d_offs.data_ptr(),
                                       stream)
        torch.cuda.synchronize()
        got_offs = d_offs.cpu().numpy().view(np.uint32)
        got_perm = d_perm.cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(got_offs, want_offs)
        untouched = np.ones(n, bool)
        untouched[: want_offs[-1]] = False
        if skip >= 0:
            untouched[want_offs[skip]:want_offs[skip + 1]] = True
        placed = ~untouched
        np.testing.assert_array_equal(got_perm[placed], want_perm[placed[: want_offs[-1]]])
        assert np.all(got_perm[untouched] == 0xFFFFFFFF)


def test_noalloc_partition_empty_input_zeroes_offsets():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d_offs = torch.full((6,), 77, dtype=torch.int32, device="cuda")
    binding.partition_keys_noalloc(0, 0, 5, -1, 0, d_offs.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert d_offs.cpu().tolist() == [0] * 6


def test_noalloc_partition_leaves_device_memory_use_unchanged():
    """After one warm-up call (which looks up the array's address and loads
    the kernels), further calls change no device allocation: the free device
    memory is the same before and after."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = 1 << 20
    keys = np.random.default_rng(3).integers(0, 16, size=n, dtype=np.uint8)
    d_keys = torch.from_numpy(keys).cuda()
    d_perm = torch.empty(n, dtype=torch.int32, device="cuda")
    d_offs = torch.empty(17, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    def call():
        binding.partition_keys_noalloc(d_keys.data_ptr(), n, 16, -1, d_perm.data_ptr(), d_offs.data_ptr(), stream)
        torch.cuda.synchronize()

    call()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    want_offs, want_perm = _expected(keys, 16)
    np.testing.assert_array_equal(d_offs.cpu().numpy().view(np.uint32), want_offs)
    np.testing.assert_array_equal(d_perm.cpu().numpy().view(np.uint32), want_perm)
