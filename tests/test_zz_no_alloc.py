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
