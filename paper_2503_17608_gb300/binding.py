"""ctypes binding of the C ABI in include/celer_gb.h.

Argument marshalling only: every step of the transport runs in the CUDA
library. There is no CPU fallback; if the library is missing or cannot be
loaded the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libceler_gb.so")

CELER_OK = 0
LOOP_HOST, LOOP_GRAPH, LOOP_PERSISTENT, LOOP_ASYNC = 0, 1, 2, 3
LOOP_NAMES = {"host": LOOP_HOST, "graph": LOOP_GRAPH, "persistent": LOOP_PERSISTENT, "async": LOOP_ASYNC}
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "capacity exceeded", 3: "CUDA error",
                4: "iteration limit reached", 5: "invalid state"}


class CelerError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class celer_material(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("Z", "A", "rho", "ne", "X0", "I")]


class celer_problem(C.Structure):
    _fields_ = [
        ("n_materials", C.c_int), ("materials", C.POINTER(celer_material)),
        ("n_layers", C.c_int), ("layer_material", C.POINTER(C.c_int)),
        ("layer_thickness", C.POINTER(C.c_double)), ("n_periods", C.c_int),
        ("half_x", C.c_double), ("half_y", C.c_double), ("Bz", C.c_double),
        ("cut_track", C.c_double), ("cut_moller", C.c_double), ("cut_brems", C.c_double),
        ("processes", C.c_int), ("tally_mode", C.c_int), ("n_zbins", C.c_int),
        ("n_slots", C.c_uint64), ("init_capacity", C.c_uint64), ("max_events", C.c_uint32),
        ("history_capacity", C.c_uint64), ("sort_policy", C.c_int), ("block_size", C.c_int),
        ("split_actions", C.c_int),
        ("seed", C.c_uint32), ("max_iterations", C.c_uint64), ("cuda_stream", C.c_void_p),
        ("field_substep_cap", C.c_int),
    ]


PRIMARY_C = np.dtype([("E", "f8"), ("pos", "f8", (3,)), ("dir", "f8", (3,)), ("ptype", "i4"), ("pad", "i4")],
                     align=True)
assert PRIMARY_C.itemsize == 64


class celer_step_stats(C.Structure):
    _fields_ = [("iteration", C.c_uint64), ("alive", C.c_uint64), ("queued", C.c_uint64), ("steps", C.c_uint64),
                ("steps_total", C.c_uint64), ("deferred", C.c_uint32), ("error", C.c_uint32),
                ("action_count", C.c_uint32 * 16)]


class celer_history(C.Structure):
    _fields_ = [("steps", C.c_uint64), ("secondaries", C.c_uint64), ("escaped", C.c_double), ("edep", C.c_double)]


HISTORY_NP = np.dtype([("steps", "u8"), ("secondaries", "u8"), ("escaped", "f8"), ("edep", "f8")], align=True)


class celer_trace_row(C.Structure):
    _fields_ = [("iteration", C.c_uint64), ("alive", C.c_uint64), ("queued", C.c_uint64), ("steps", C.c_uint64),
                ("action_count", C.c_uint32 * 16)]


class celer_request(C.Structure):
    _fields_ = [("arrival_s", C.c_double), ("event", C.c_uint32), ("pad", C.c_uint32),
                ("primaries", C.c_void_p), ("n", C.c_uint64)]


class celer_request_result(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("arrival_s", "admit_s", "done_s", "edep", "escaped")]


REQUEST_RESULT_NP = np.dtype([(k, "f8") for k in ("arrival_s", "admit_s", "done_s", "edep", "escaped")])


class celer_serve_options(C.Structure):
    _fields_ = [("mode", C.c_int), ("chunk_iterations", C.c_uint64), ("footprint_per_primary", C.c_double),
                ("max_in_flight", C.c_uint32), ("stop_admitting_s", C.c_double),
                ("tallies_out", C.POINTER(C.c_double))]


class celer_serve_summary(C.Structure):
    _fields_ = [("wall_s", C.c_double), ("track_steps", C.c_uint64), ("admitted", C.c_uint64),
                ("completed", C.c_uint64), ("chunks", C.c_uint64)]


class celer_tune_trial(C.Structure):
    _fields_ = [("n_slots", C.c_uint64), ("block_size", C.c_int), ("sort_policy", C.c_int), ("mode", C.c_int),
                ("track_steps_per_s", C.c_double), ("ms", C.c_double), ("async_warps", C.c_int)]


ACTION_NAMES = ["none", "zup", "zdown", "side", "range", "trapped", "compton", "photoelectric", "pair", "moller",
                "brems", "field"]

# Every entry point declared in include/celer_gb.h.
EXPORTS = [
    "celer_status_string", "celer_last_error", "celer_create", "celer_destroy", "celer_add_primaries",
    "celer_add_primaries_device",
    "celer_step", "celer_run_events", "celer_read_tallies", "celer_reset_event", "celer_event_live",
    "celer_read_history", "celer_get_stats", "celer_set_sort_policy", "celer_set_split_actions", "celer_read_trace",
    "celer_read_loop_profile",
    "celer_enable_kernel_timing", "celer_kernel_timing", "celer_debug_partition", "celer_debug_table",
    "celer_debug_philox", "celer_debug_curand_philox", "celer_partition_keys_noalloc", "celer_debug_math",
    "celer_run_iterations", "celer_read_event_live", "celer_serve", "celer_autotune", "celer_get_problem",
    "celer_debug_sample", "celer_debug_slots", "celer_set_hit_readout", "celer_set_grid_blocks",
    "celer_set_parent_reuse", "celer_set_async_warps", "celer_debug_barrier_timeout", "celer_debug_queue_wait",
    "celer_debug_tracks", "celer_debug_fp64_rate", "celer_debug_lane_counts",
]

_lib = None


def load(path: Optional[str] = None):
    """Load libceler_gb.so (built by paper_2503_17608_gb300.build). Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run paper_2503_17608_gb300.build.build())")
    L = C.CDLL(path)
    vp, u64, u32, i32, dp = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int, C.POINTER(C.c_double)
    sigs = {
        "celer_status_string": ([i32], C.c_char_p),
        "celer_last_error": ([vp], C.c_char_p),
        "celer_create": ([C.POINTER(celer_problem), C.POINTER(vp)], i32),
        "celer_destroy": ([vp], None),
        "celer_add_primaries": ([vp, u32, vp, u64], i32),
        "celer_add_primaries_device": ([vp, u32, vp, u64], i32),
        "celer_step": ([vp, C.POINTER(celer_step_stats)], i32),
        "celer_run_events": ([vp, i32], i32),
        "celer_read_tallies": ([vp, u32, dp, u64, dp], i32),
        "celer_reset_event": ([vp, u32], i32),
        "celer_event_live": ([vp, u32, C.POINTER(u64)], i32),
        "celer_read_history": ([vp, u64, u64, vp, dp], i32),
        "celer_get_stats": ([vp, C.POINTER(celer_step_stats)], i32),
        "celer_set_sort_policy": ([vp, i32], i32),
        "celer_set_split_actions": ([vp, i32], i32),
        "celer_read_loop_profile": ([vp, C.POINTER(u64), i32], i32),
        "celer_read_trace": ([vp, vp, u64, C.POINTER(u64)], i32),
        "celer_enable_kernel_timing": ([vp, i32], i32),
        "celer_kernel_timing": ([vp, C.POINTER(C.c_char_p), dp, C.POINTER(u64), i32, C.POINTER(i32)], i32),
        "celer_debug_partition": ([vp, vp, vp, vp, C.POINTER(i32), C.POINTER(i32)], i32),
        "celer_debug_table": ([vp, i32, i32, dp], i32),
        "celer_debug_philox": ([vp, vp, u64], i32),
        "celer_debug_math": ([i32, vp, u64, vp], i32),
        "celer_debug_curand_philox": ([u64, u64, u64, vp, u64], i32),
        "celer_debug_sample": ([i32, u32, u32, vp, C.c_double, vp, vp, u64, vp, vp, vp, vp], i32),
        "celer_debug_slots": ([vp, vp, vp, C.POINTER(i32)], i32),
        "celer_set_hit_readout": ([vp, i32, vp, u64], i32),
        "celer_set_grid_blocks": ([vp, i32], i32),
        "celer_set_parent_reuse": ([vp, i32], i32),
        "celer_set_async_warps": ([vp, i32], i32),
        "celer_debug_barrier_timeout": ([i32, i32, u64, C.POINTER(u32), C.POINTER(u32)], i32),
        "celer_debug_queue_wait": ([i32, u64, C.POINTER(u32), C.POINTER(u32)], i32),
        "celer_debug_tracks": ([vp, vp, vp, vp, vp], i32),
        "celer_partition_keys_noalloc": ([vp, u64, i32, i32, vp, vp, vp], i32),
        "celer_debug_fp64_rate": ([i32, u64, C.POINTER(C.c_double), C.POINTER(C.c_double)], i32),
        "celer_debug_lane_counts": ([vp, i32, C.POINTER(C.c_int)], i32),
        "celer_run_iterations": ([vp, i32, u64, C.POINTER(u64)], i32),
        "celer_read_event_live": ([vp, u32, u32, vp], i32),
        "celer_serve": ([vp, vp, u64, C.POINTER(celer_serve_options), vp, C.POINTER(celer_serve_summary)], i32),
        "celer_autotune": ([C.POINTER(celer_problem), vp, vp, u64, vp, i32, vp, i32, vp, i32, vp, i32, vp, i32,
                            C.POINTER(i32), C.POINTER(celer_tune_trial)], i32),
        "celer_get_problem": ([vp, C.POINTER(celer_problem)], i32),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(status, ctx=None):
    if status != CELER_OK:
        msg = ""
        if ctx:
            msg = (load().celer_last_error(ctx) or b"").decode()
        raise CelerError(status, msg)


def to_c_primaries(primaries: np.ndarray, out: Optional[np.ndarray] = None) -> np.ndarray:
    n = len(primaries)
    p = out if out is not None else np.zeros(n, dtype=PRIMARY_C)
    p["E"] = primaries["E"]
    p["pos"] = primaries["pos"]
    p["dir"] = primaries["dir"]
    p["ptype"] = primaries["ptype"]
    return p


def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover - torch without CUDA
        pass
    return None


class ProblemStruct:
    """A celer_problem filled from a workloads.Problem; keeps its arrays alive."""

    def __init__(self, prob: wl.Problem, stream=None, max_iterations: int = 0):
        self._mats = (celer_material * len(prob.materials))(
            *[celer_material(m.Z, m.A, m.rho, m.ne, m.X0, m.I) for m in prob.materials])
        self._lm = (C.c_int * len(prob.layer_material))(*prob.layer_material)
        self._lt = (C.c_double * len(prob.layer_thickness))(*prob.layer_thickness)
        cp = celer_problem()
        cp.n_materials = len(prob.materials)
        cp.materials = self._mats
        cp.n_layers = len(prob.layer_material)
        cp.layer_material = self._lm
        cp.layer_thickness = self._lt
        cp.n_periods = prob.n_periods
        cp.half_x, cp.half_y, cp.Bz = prob.half_x, prob.half_y, prob.Bz
        cp.cut_track, cp.cut_moller, cp.cut_brems = prob.cut_track, prob.cut_moller, prob.cut_brems
        cp.processes, cp.tally_mode, cp.n_zbins = prob.processes, prob.tally_mode, prob.n_zbins
        cp.n_slots, cp.init_capacity = prob.n_slots, prob.init_capacity
        cp.max_events, cp.history_capacity = prob.max_events, prob.history_capacity
        cp.sort_policy, cp.block_size, cp.seed = prob.sort_policy, prob.block_size, prob.seed
        cp.split_actions = prob.split_actions
        cp.max_iterations = max_iterations
        cp.cuda_stream = stream
        cp.field_substep_cap = prob.field_substep_cap
        self.c = cp


class Context:
    """A transport context built from a workloads.Problem."""

    def __init__(self, prob: wl.Problem, stream=None, max_iterations: int = 0):
        L = load()
        self.prob = prob
        self.n_bins = prob.n_bins
        self.stream = stream if stream is not None else _torch_stream()
        self._ps = ProblemStruct(prob, self.stream, max_iterations)
        cp = self._ps.c
        h = C.c_void_p()
        _check(L.celer_create(C.byref(cp), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().celer_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- transport
    def add_primaries(self, event: int, primaries: np.ndarray):
        p = primaries if primaries.dtype == PRIMARY_C else to_c_primaries(primaries)
        p = np.ascontiguousarray(p)
        _check(load().celer_add_primaries(self._h, int(event), p.ctypes.data, len(p)), self._h)

    def add_primaries_device(self, event: int, device_ptr: int, n: int):
        """Queue n celer_primary records already in device memory (e.g. the
        data_ptr() of a CUDA tensor holding 64-byte records)."""
        _check(load().celer_add_primaries_device(self._h, int(event), C.c_void_p(int(device_ptr)), int(n)), self._h)

    def add_events(self, primaries: np.ndarray):
        """Queue primaries grouped by their event field, in order of first appearance."""
        ev = primaries["event"]
        for e in dict.fromkeys(ev.tolist()):
            self.add_primaries(e, primaries[ev == e])

    def step(self):
        s = celer_step_stats()
        _check(load().celer_step(self._h, C.byref(s)), self._h)
        return _stats_dict(s)

    def step_async(self):
        _check(load().celer_step(self._h, None), self._h)

    def run_events(self, mode=LOOP_GRAPH, use_graph=None):
        """Step until done. mode: LOOP_HOST, LOOP_GRAPH, LOOP_PERSISTENT or
        LOOP_ASYNC (block-pass policies only; use_graph=True/False is accepted
        as LOOP_GRAPH/LOOP_HOST)."""
        if use_graph is not None:
            mode = LOOP_GRAPH if use_graph else LOOP_HOST
        _check(load().celer_run_events(self._h, int(mode)), self._h)

    def loop_profile(self):
        """Persistent-loop profile in SM cycles: per phase (block 0 view, with
        barrier waits), slowest block's work per phase, bookkeeping."""
        out = (C.c_uint64 * 10)()
        _check(load().celer_read_loop_profile(self._h, out, 10), self._h)
        v = list(out)
        names = ("fill_step", "scatter", "step")
        return dict(phase={k: v[i] for i, k in enumerate(names)},
                    slowest_work={k: v[4 + i] for i, k in enumerate(names)},
                    bookkeeping={"fill_step": v[8], "step": v[9]})

    def run_iterations(self, mode=LOOP_PERSISTENT, budget: int = 0) -> int:
        done = C.c_uint64()
        _check(load().celer_run_iterations(self._h, int(mode), int(budget), C.byref(done)), self._h)
        return done.value

    def event_live_rows(self, first: int = 0, count: int = None):
        count = self.prob.max_events - first if count is None else count
        out = np.zeros(count, np.uint32)
        _check(load().celer_read_event_live(self._h, first, count, out.ctypes.data), self._h)
        return out

    def serve(self, requests, mode=LOOP_PERSISTENT, chunk_iterations=16, footprint_per_primary=40.0,
              max_in_flight=0, stop_admitting_s=0.0, with_tallies=False):
        """Continuous batching. requests: list of (arrival_s, event_id, primaries)
        in arrival order. Returns (results ndarray, summary dict, tallies or None)."""
        n = len(requests)
        keep = [np.ascontiguousarray(to_c_primaries(p)) for _, _, p in requests]
        reqs = (celer_request * max(n, 1))()
        for i, ((t, ev, _), arr) in enumerate(zip(requests, keep)):
            reqs[i].arrival_s = float(t)
            reqs[i].event = int(ev)
            reqs[i].primaries = arr.ctypes.data
            reqs[i].n = len(arr)
        res = np.zeros(max(n, 1), dtype=REQUEST_RESULT_NP)
        tallies = np.zeros((max(n, 1), self.n_bins)) if with_tallies else None
        opt = celer_serve_options()
        opt.mode, opt.chunk_iterations, opt.footprint_per_primary = int(mode), chunk_iterations, footprint_per_primary
        opt.max_in_flight, opt.stop_admitting_s = max_in_flight, stop_admitting_s
        opt.tallies_out = tallies.ctypes.data_as(C.POINTER(C.c_double)) if with_tallies else None
        summ = celer_serve_summary()
        _check(load().celer_serve(self._h, C.cast(reqs, C.c_void_p), n, C.byref(opt), res.ctypes.data,
                                  C.byref(summ)), self._h)
        summary = dict(wall_s=summ.wall_s, track_steps=summ.track_steps, admitted=summ.admitted,
                       completed=summ.completed, chunks=summ.chunks)
        return res[:n], summary, (tallies[:n] if with_tallies else None)

    def set_split_actions(self, split: bool):
        _check(load().celer_set_split_actions(self._h, 1 if split else 0), self._h)

    def read_tallies(self, event: int = 0):
        out = np.zeros(self.n_bins)
        esc = C.c_double()
        _check(load().celer_read_tallies(self._h, int(event), out.ctypes.data_as(C.POINTER(C.c_double)),
                                         self.n_bins, C.byref(esc)), self._h)
        return out, esc.value

    def reset_event(self, event: int):
        _check(load().celer_reset_event(self._h, int(event)), self._h)

    def event_live(self, event: int) -> int:
        v = C.c_uint64()
        _check(load().celer_event_live(self._h, int(event), C.byref(v)), self._h)
        return v.value

    def read_history(self, first: int, count: int, with_edep: bool = True):
        hist = np.zeros(count, dtype=HISTORY_NP)
        edep = np.zeros((count, self.n_bins)) if with_edep else None
        _check(load().celer_read_history(self._h, first, count, hist.ctypes.data,
                                         edep.ctypes.data_as(C.POINTER(C.c_double)) if with_edep else None),
               self._h)
        return hist, edep

    def stats(self):
        s = celer_step_stats()
        _check(load().celer_get_stats(self._h, C.byref(s)), self._h)
        return _stats_dict(s)

    def set_hit_readout(self, mode: int, host_hits=None):
        """Per-iteration copy of the tally rows into host_hits during host-loop
        runs: mode 0 off, 1 stream-ordered, 2 synchronous. host_hits: a pinned
        float64 torch tensor (or array) of at least max_events x bins."""
        if mode == 0:
            _check(load().celer_set_hit_readout(self._h, 0, None, 0), self._h)
            self._hits = None
            return
        ptr = host_hits.data_ptr() if hasattr(host_hits, "data_ptr") else host_hits.ctypes.data
        n = host_hits.numel() if hasattr(host_hits, "numel") else host_hits.size
        _check(load().celer_set_hit_readout(self._h, int(mode), C.c_void_p(ptr), int(n)), self._h)
        self._hits = host_hits  # keep it alive while the mode is on

    def set_parent_reuse(self, on: bool):
        """A pair's first photon starts in the converted photon's slot."""
        _check(load().celer_set_parent_reuse(self._h, int(bool(on))), self._h)

    def set_async_warps(self, on: bool):
        """Asynchronous loop, block-local policy: per-warp scheduling from the
        block's queues (True) or block passes (False)."""
        _check(load().celer_set_async_warps(self._h, int(bool(on))), self._h)

    def set_grid_blocks(self, blocks: int):
        """Cap the GPU blocks of this context's kernels (0: one per SM)."""
        _check(load().celer_set_grid_blocks(self._h, int(blocks)), self._h)

    def set_sort_policy(self, policy: int):
        _check(load().celer_set_sort_policy(self._h, int(policy)), self._h)

    def trace(self, n_max: int = 1 << 16):
        rows = (celer_trace_row * n_max)()
        n = C.c_uint64()
        _check(load().celer_read_trace(self._h, C.cast(rows, C.c_void_p), n_max, C.byref(n)), self._h)
        return [dict(iteration=r.iteration, alive=r.alive, queued=r.queued, steps=r.steps,
                     actions=list(r.action_count)[:len(ACTION_NAMES)]) for r in rows[:n.value]]

    def enable_kernel_timing(self, enable: bool = True):
        _check(load().celer_enable_kernel_timing(self._h, 1 if enable else 0), self._h)

    def kernel_timing(self):
        n_max = 32
        names = (C.c_char_p * n_max)()
        tot = (C.c_double * n_max)()
        cnt = (C.c_uint64 * n_max)()
        n = C.c_int()
        _check(load().celer_kernel_timing(self._h, names, tot, cnt, n_max, C.byref(n)), self._h)
        return {names[i].decode(): dict(total_ms=tot[i], launches=cnt[i]) for i in range(n.value)}

    # -- diagnostics
    def debug_partition(self):
        N = self.prob.n_slots
        keys = np.zeros(N, np.uint8)
        perm = np.zeros(N, np.uint32)
        offs = np.zeros(17, np.uint32)
        nk = C.c_int()
        nb = C.c_int()
        _check(load().celer_debug_partition(self._h, keys.ctypes.data, perm.ctypes.data, offs.ctypes.data,
                                            C.byref(nk), C.byref(nb)), self._h)
        self.partition_blocks = nb.value
        return keys, perm, offs[:nk.value + 1]

    def debug_slots(self):
        """Per-slot status and particle type (device state, host copies)."""
        n = self.prob.n_slots
        status = np.zeros(n, np.uint8)
        ptype = np.zeros(n, np.uint8)
        nb = C.c_int()
        _check(load().celer_debug_slots(self._h, status.ctypes.data, ptype.ctypes.data, C.byref(nb)), self._h)
        self._loop_blocks = nb.value
        return dict(status=status, ptype=ptype)

    def debug_tracks(self):
        """Per-slot track id, event, layer and state (x, y, z, ux, uy, uz, E)."""
        n = self.prob.n_slots
        tid = np.zeros(n, np.uint64)
        event = np.zeros(n, np.uint32)
        layer = np.zeros(n, np.int32)
        state = np.zeros((7, n), np.float64)
        _check(load().celer_debug_tracks(self._h, tid.ctypes.data, event.ctypes.data, layer.ctypes.data,
                                         state.ctypes.data), self._h)
        return dict(tid=tid, event=event, layer=layer, pos=state[0:3].T.copy(), dir=state[3:6].T.copy(),
                    E=state[6].copy())

    def loop_blocks(self) -> int:
        """GPU blocks of the block-pass policies (block b owns chunks b, b + B, ...)."""
        if getattr(self, "_loop_blocks", None) is None:
            self.debug_slots()
        return self._loop_blocks

    def debug_table(self, mat: int, col: int):
        out = np.zeros(200)
        _check(load().celer_debug_table(self._h, mat, col, out.ctypes.data_as(C.POINTER(C.c_double))), self._h)
        return out


def _stats_dict(s):
    return dict(iteration=s.iteration, alive=s.alive, queued=s.queued, steps=s.steps, steps_total=s.steps_total,
                deferred=s.deferred, error=s.error, actions=list(s.action_count)[:len(ACTION_NAMES)])


def partition_keys_noalloc(d_keys: int, n: int, n_keys: int, skip_key: int, d_perm: int, d_offsets: int,
                           stream=None):
    """Stable partition of 0..n-1 by key into device buffers, using only the
    library's fixed working array (no device allocation). Pointers are device
    addresses (e.g. tensor.data_ptr())."""
    _check(load().celer_partition_keys_noalloc(C.c_void_p(d_keys), n, n_keys, skip_key, C.c_void_p(d_perm),
                                               C.c_void_p(d_offsets), C.c_void_p(stream) if stream else None))


def debug_fp64_rate(blocks_per_sm: int = 4, iters: int = 40000):
    """Measured FP64 fused multiply-add throughput of the device (TFLOP/s)
    and the timed launch's milliseconds."""
    tf, ms = C.c_double(), C.c_double()
    _check(load().celer_debug_fp64_rate(blocks_per_sm, iters, C.byref(tf), C.byref(ms)))
    return tf.value, ms.value


LANE_SITES = ["piece g_geom", "piece e_geom", "piece e_range", "piece compton", "piece pe", "piece pair",
              "piece moller", "piece brems", "fill", "step_limit", "along", "compton", "photoelectric", "pair",
              "moller", "brems", "compton_attempt", "moller_attempt", "helix_side", "idle",
              "photon_crossing: claim", "photon_crossing: step", "photon_crossing: next limit",
              "electron_crossing: claim", "electron_crossing: step", "electron_crossing: next limit",
              "photon limit: loads", "photon limit: grid (log)", "photon limit: cross sections",
              "photon limit: planes", "photon limit: rest and stores", "queue push",
              "compton: claim", "compton: step", "compton: next limit"]


def debug_lane_counts():
    """Visits, summed active lanes and summed SM cycles (timed sites) per
    instrumented site since the last read (the diagnostic build only):
    {site: (visits, lanes, cycles)}."""
    out = np.zeros(3 * len(LANE_SITES), dtype=np.uint64)
    n = C.c_int()
    _check(load().celer_debug_lane_counts(out.ctypes.data, len(LANE_SITES), C.byref(n)))
    return {name: (int(out[3 * k]), int(out[3 * k + 1]), int(out[3 * k + 2]))
            for k, name in enumerate(LANE_SITES[:n.value])}


def autotune(prob: wl.Problem, primaries: np.ndarray, slot_counts, block_sizes, policies, modes, stream=None):
    """Measure every combination on the sample; returns (best, trials) as dicts."""
    ps = ProblemStruct(prob, stream if stream is not None else _torch_stream())
    cprim = np.ascontiguousarray(to_c_primaries(primaries))
    events = np.ascontiguousarray(primaries["event"].astype(np.uint32))
    sc = (C.c_uint64 * len(slot_counts))(*slot_counts)
    bs = (C.c_int * len(block_sizes))(*block_sizes)
    po = (C.c_int * len(policies))(*policies)
    mo = (C.c_int * len(modes))(*modes)
    n_max = 2 * len(slot_counts) * len(block_sizes) * len(policies) * len(modes)  # local + async: two schedules
    trials = (celer_tune_trial * n_max)()
    n_out = C.c_int()
    best = celer_tune_trial()
    _check(load().celer_autotune(C.byref(ps.c), cprim.ctypes.data, events.ctypes.data, len(cprim), sc, len(sc), bs,
                                 len(bs), po, len(po), mo, len(mo), trials, n_max, C.byref(n_out), C.byref(best)))

    def d(t):
        return dict(n_slots=t.n_slots, block_size=t.block_size, sort_policy=t.sort_policy, mode=t.mode,
                    track_steps_per_s=t.track_steps_per_s, ms=t.ms, async_warps=t.async_warps)

    return d(best), [d(trials[i]) for i in range(n_out.value)]


def debug_philox(ctr_key: np.ndarray) -> np.ndarray:
    """Device Philox4x32-10 on rows (c0, c1, c2, c3, k0, k1)."""
    a = np.ascontiguousarray(ctr_key, dtype=np.uint32)
    out = np.zeros((len(a), 4), np.uint32)
    _check(load().celer_debug_philox(a.ctypes.data, out.ctypes.data, len(a)))
    return out


def debug_math(fn: int, x: np.ndarray) -> np.ndarray:
    """Device elementary function fn on x: 0/1 table-driven log/exp, 2/3 CUDA
    log/exp, 4/5 table-driven sin/cos of 2 pi x, 6/7 CUDA sin/cos of 2 pi x,
    8/9 table-driven sin/cos of x, 10/11 CUDA sin/cos of x."""
    a = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros_like(a)
    _check(load().celer_debug_math(int(fn), a.ctypes.data, len(a), out.ctypes.data))
    return out


def debug_curand_philox(seed: int, subsequence: int, offset4: int, n: int) -> np.ndarray:
    out = np.zeros((n, 4), np.uint32)
    _check(load().celer_debug_curand_philox(seed, subsequence, offset4, out.ctypes.data, n))
    return out

def debug_sample(which: int, E: np.ndarray, tid: np.ndarray, ctr: np.ndarray, seed: int = 20250321, event: int = 0,
                 cut: float = 1.0):
    """Device rejection samplers: which 0 filtered Compton, 1 plain FP64
    Compton, 2 filtered Moller, 3 plain FP64 Moller. Returns eps, cos(theta)
    (Compton), the draw counter after sampling and the ok flags."""
    e = np.ascontiguousarray(E, dtype=np.float64)
    t = np.ascontiguousarray(tid, dtype=np.uint64)
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    n = len(e)
    eps = np.zeros(n)
    cost = np.zeros(n)
    ctr_out = np.zeros(n, np.uint32)
    ok = np.zeros(n, np.uint8)
    _check(load().celer_debug_sample(int(which), C.c_uint32(seed), C.c_uint32(event), e.ctypes.data, C.c_double(cut),
                                     t.ctypes.data, c.ctypes.data, C.c_uint64(n), eps.ctypes.data, cost.ctypes.data,
                                     ctr_out.ctypes.data, ok.ctypes.data))
    return eps, cost, ctr_out, ok


def debug_barrier_timeout(blocks: int, absent_block: int, timeout_cycles: int):
    """Bounded grid-barrier wait with one block that never arrives: returns
    (status, error bits, abort word); status 4 (CELER_ERR_TIMEOUT) when the
    waiting blocks gave up as they should."""
    err = C.c_uint32()
    ab = C.c_uint32()
    st = load().celer_debug_barrier_timeout(int(blocks), int(absent_block), C.c_uint64(timeout_cycles), C.byref(err),
                                            C.byref(ab))
    return st, err.value, ab.value


def debug_queue_wait(which: int, timeout_cycles: int):
    """Bounded wait of the asynchronous loop for a buffer entry (which 0, 2)
    or a shared-memory queue entry (1, 3) that nothing writes (0, 1) or that
    was written first (2, 3): returns (status, error bits, abort word)."""
    err = C.c_uint32()
    ab = C.c_uint32()
    st = load().celer_debug_queue_wait(int(which), C.c_uint64(timeout_cycles), C.byref(err), C.byref(ab))
    return st, err.value, ab.value
