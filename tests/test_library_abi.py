"""The CUDA library loads and exports every entry point declared in
include/*.h (CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

from paper_2503_17608_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(celer_[a-z0-9_]+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("celer_create", "celer_add_primaries", "celer_step", "celer_run_events", "celer_read_tallies"):
        assert required in names


def test_library_exports_every_declared_symbol():
    build.build()
    lib = ctypes.CDLL(binding.LIB_PATH)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(binding.EXPORTS) == declared_symbols()


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(RuntimeError):
        binding._lib = None
        saved = binding._lib
        try:
            binding.load(str(tmp_path / "missing.so"))
        finally:
            binding._lib = saved


def test_status_strings():
    lib = binding.load()
    assert lib.celer_status_string(0) == b"ok"
    assert lib.celer_status_string(2) == b"capacity exceeded"


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++17")])
def test_header_is_plain_c(tmp_path, lang, std):
    """The boundary header compiles on its own as C99 and as C++ (no torch
    or CUDA types in the signatures)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / ("use." + ("c" if lang == "c" else "cpp"))
    src.write_text('#include "celer_gb.h"\nint main(void) { celer_tune_trial t; (void)t; return 0; }\n')
    r = subprocess.run([cc, std, "-Wall", "-Werror", "-fsyntax-only", "-I", os.path.join(ROOT, "include"), str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_argument_checks_before_any_device_call():
    """Calls with a null context or out-of-range arguments return
    CELER_ERR_INVALID from the host-side checks, before the device is
    touched (so they run here, with no GPU)."""
    import ctypes as C

    lib = binding.load()
    u32 = C.c_uint32()
    INVALID = 1
    assert lib.celer_set_async_warps(None, 1) == INVALID
    assert lib.celer_set_parent_reuse(None, 1) == INVALID
    assert lib.celer_set_grid_blocks(None, 2) == INVALID
    assert lib.celer_run_events(None, binding.LOOP_ASYNC) == INVALID
    assert lib.celer_run_iterations(None, binding.LOOP_ASYNC, 4, None) == INVALID
    for which, timeout in ((-1, 1000), (4, 1000), (0, 0), (1, 5_000_000_000)):
        assert lib.celer_debug_queue_wait(which, C.c_uint64(timeout), C.byref(u32), C.byref(u32)) == INVALID
    assert lib.celer_debug_queue_wait(0, C.c_uint64(1000), None, None) == INVALID
    for args in ((1, 0, 1000), (9, 0, 1000), (4, 4, 1000), (4, -2, 1000), (4, 0, 0)):
        blocks, absent, timeout = args
        assert lib.celer_debug_barrier_timeout(blocks, absent, C.c_uint64(timeout), C.byref(u32),
                                               C.byref(u32)) == INVALID
    assert lib.celer_debug_tracks(None, None, None, None, None) == INVALID
