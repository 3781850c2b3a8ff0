"""Python access to the CPU oracle (test infrastructure only).

The oracle is a plain history-based transport in C (see oracle.h). Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
use it; the product path never imports this package.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

OM_NGRID = 200
COL_COMPTON, COL_PE, COL_PAIR, COL_MOLLER, COL_BREMS, COL_DEDX, COL_RANGE = range(7)
SEL_COMPTON, SEL_PE, SEL_PAIR, SEL_MOLLER, SEL_BREMS = range(5)


class om_material(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("Z", "A", "rho", "ne", "X0", "I")]


class om_problem(C.Structure):
    _fields_ = [
        ("n_materials", C.c_int), ("materials", C.POINTER(om_material)),
        ("n_layers", C.c_int), ("layer_material", C.POINTER(C.c_int)),
        ("layer_thickness", C.POINTER(C.c_double)), ("n_periods", C.c_int),
        ("half_x", C.c_double), ("half_y", C.c_double), ("Bz", C.c_double),
        ("cut_track", C.c_double), ("cut_moller", C.c_double), ("cut_brems", C.c_double),
        ("processes", C.c_int), ("tally_mode", C.c_int), ("n_zbins", C.c_int),
        ("seed", C.c_uint32), ("field_substep_cap", C.c_int),
    ]


class om_primary(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("E", "x", "y", "z", "ux", "uy", "uz")] + [
        ("ptype", C.c_int32), ("event", C.c_uint32), ("tid", C.c_uint64)]


class om_history(C.Structure):
    _fields_ = [("steps", C.c_uint64), ("secondaries", C.c_uint64),
                ("escaped", C.c_double), ("path", C.c_double)]


class om_rng(C.Structure):
    _fields_ = [("seed", C.c_uint32), ("event", C.c_uint32), ("tid", C.c_uint64), ("ctr", C.c_uint32)]


class om_track(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("E", "x", "y", "z", "ux", "uy", "uz", "nmfp")] + [
        ("ptype", C.c_int32), ("layer", C.c_int32), ("tid", C.c_uint64), ("ctr", C.c_uint32)]


PRIMARY_NP = np.dtype([("E", "f8"), ("x", "f8"), ("y", "f8"), ("z", "f8"), ("ux", "f8"), ("uy", "f8"),
                       ("uz", "f8"), ("ptype", "i4"), ("event", "u4"), ("tid", "u8")], align=True)
HISTORY_NP = np.dtype([("steps", "u8"), ("secondaries", "u8"), ("escaped", "f8"), ("path", "f8")],
                      align=True)

_dp = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.om_world_create.restype = C.c_void_p
        L.om_world_create.argtypes = [C.POINTER(om_problem), C.c_char_p, C.c_int]
        L.om_world_destroy.argtypes = [C.c_void_p]
        L.om_world_nbins.argtypes = [C.c_void_p]
        L.om_world_nlayers.argtypes = [C.c_void_p]
        L.om_world_boundaries.argtypes = [C.c_void_p, _dp]
        L.om_world_table.argtypes = [C.c_void_p, C.c_int, C.c_int, _dp]
        L.om_world_lookup.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double]
        L.om_world_lookup.restype = C.c_double
        L.om_world_inv_range.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.om_world_inv_range.restype = C.c_double
        L.om_world_grid.argtypes = [C.c_void_p, _dp]
        L.om_world_initial_layer.argtypes = [C.c_void_p, C.c_double, C.c_double]
        L.om_run.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_int, C.c_void_p, _dp]
        L.om_transport_track.argtypes = [C.c_void_p, C.c_uint32, C.POINTER(om_track), C.c_uint64,
                                         C.POINTER(C.c_uint64), _dp, _dp, _dp, C.POINTER(C.c_uint64)]
        L.om_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.om_raw_word.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint32]
        L.om_raw_word.restype = C.c_uint64
        L.om_uniform.argtypes = [C.c_uint64]
        L.om_uniform.restype = C.c_double
        L.om_draw.argtypes = [C.POINTER(om_rng)]
        L.om_draw.restype = C.c_double
        L.om_draw_raw.argtypes = [C.POINTER(om_rng)]
        L.om_draw_raw.restype = C.c_uint64
        for name, args in (("om_sigma_kn", [C.c_double]), ("om_sigma_moller", [C.c_double, C.c_double]),
                           ("om_dedx_collision", [C.c_double] * 4)):
            getattr(L, name).argtypes = args
            getattr(L, name).restype = C.c_double
        L.om_electron_density.argtypes = [C.POINTER(om_material)]
        L.om_electron_density.restype = C.c_double
        L.om_gauss_legendre.argtypes = [C.c_int, _dp, _dp]
        L.om_sample_compton.argtypes = [C.c_double, C.POINTER(om_rng), _dp, _dp]
        L.om_sample_moller.argtypes = [C.c_double, C.c_double, C.POINTER(om_rng)]
        L.om_sample_moller.restype = C.c_double
        L.om_sample_brems.argtypes = [C.c_double, C.c_double, C.POINTER(om_rng)]
        L.om_sample_brems.restype = C.c_double
        L.om_sample_isotropic.argtypes = [C.POINTER(om_rng), _dp]
        L.om_rotate.argtypes = [_dp, C.c_double, C.c_double, _dp]
        L.om_helix_move.argtypes = [C.c_double, C.c_double, _dp, _dp]
        L.om_rk_move.argtypes = [C.c_double, C.c_double, C.c_int, _dp, _dp]
        L.om_rk_substeps.argtypes = [C.c_double, C.c_double]
        L.om_rk_substeps.restype = C.c_int
        L.om_helix_side_distance.argtypes = [C.c_double, _dp, _dp, C.c_double, C.c_double, C.POINTER(C.c_int)]
        L.om_helix_side_distance.restype = C.c_double
        L.om_curvature.argtypes = [C.c_int, C.c_double, C.c_double]
        L.om_curvature.restype = C.c_double
        L.om_select_process.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double]
        L.om_select_process.restype = C.c_int
        _lib = L
    return _lib


def _arr(a, ctype=C.c_double):
    return a.ctypes.data_as(C.POINTER(ctype))


class World:
    """An oracle geometry + physics tables built from a workloads.Problem."""

    def __init__(self, prob):
        L = lib()
        self.prob = prob
        self._mats = (om_material * len(prob.materials))(
            *[om_material(m.Z, m.A, m.rho, m.ne, m.X0, m.I) for m in prob.materials])
        self._lm = (C.c_int * len(prob.layer_material))(*prob.layer_material)
        self._lt = (C.c_double * len(prob.layer_thickness))(*prob.layer_thickness)
        p = om_problem()
        p.n_materials = len(prob.materials)
        p.materials = self._mats
        p.n_layers = len(prob.layer_material)
        p.layer_material = self._lm
        p.layer_thickness = self._lt
        p.n_periods = prob.n_periods
        p.half_x, p.half_y, p.Bz = prob.half_x, prob.half_y, prob.Bz
        p.cut_track, p.cut_moller, p.cut_brems = prob.cut_track, prob.cut_moller, prob.cut_brems
        p.processes, p.tally_mode, p.n_zbins = prob.processes, prob.tally_mode, prob.n_zbins
        p.seed = prob.seed
        p.field_substep_cap = prob.field_substep_cap
        err = C.create_string_buffer(256)
        self._h = L.om_world_create(C.byref(p), err, 256)
        if not self._h:
            raise ValueError(err.value.decode())
        self.nbins = L.om_world_nbins(self._h)
        self.nlayers = L.om_world_nlayers(self._h)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().om_world_destroy(self._h)
            self._h = None

    def boundaries(self):
        out = np.zeros(self.nlayers + 1)
        lib().om_world_boundaries(self._h, _arr(out))
        return out

    def table(self, mat, col):
        out = np.zeros(OM_NGRID)
        lib().om_world_table(self._h, mat, col, _arr(out))
        return out

    def grid(self):
        out = np.zeros(OM_NGRID)
        lib().om_world_grid(self._h, _arr(out))
        return out

    def lookup(self, mat, col, E):
        return lib().om_world_lookup(self._h, mat, col, float(E))

    def inv_range(self, mat, r):
        return lib().om_world_inv_range(self._h, mat, float(r))

    def select_process(self, mat, ptype, E, u):
        return lib().om_select_process(self._h, mat, ptype, float(E), float(u))

    def run(self, primaries, n_threads=None, with_edep=True):
        """Transport primaries (workloads.PRIMARY_DTYPE); returns (hist, edep).
        Each primary's track id is its index within its event, in order."""
        n = len(primaries)
        if n_threads is None:
            n_threads = max(1, len(os.sched_getaffinity(0)))
        pr = np.zeros(n, dtype=PRIMARY_NP)
        pr["E"] = primaries["E"]
        pr["x"], pr["y"], pr["z"] = primaries["pos"][:, 0], primaries["pos"][:, 1], primaries["pos"][:, 2]
        pr["ux"], pr["uy"], pr["uz"] = primaries["dir"][:, 0], primaries["dir"][:, 1], primaries["dir"][:, 2]
        pr["ptype"] = primaries["ptype"]
        pr["event"] = primaries["event"]
        pr["tid"] = primary_track_ids(primaries["event"])
        hist = np.zeros(n, dtype=HISTORY_NP)
        edep = np.zeros((n, self.nbins)) if with_edep else None
        lib().om_run(self._h, pr.ctypes.data, n, int(n_threads), hist.ctypes.data,
                     _arr(edep) if with_edep else None)
        return hist, edep

    def transport_track(self, E, pos, direction, ptype, tid=0, event=0, max_steps=10**7, layer=None):
        t = om_track()
        t.E = E
        t.x, t.y, t.z = pos
        t.ux, t.uy, t.uz = direction
        t.nmfp = -1.0
        t.ptype = ptype
        t.layer = lib().om_world_initial_layer(self._h, pos[2], direction[2]) if layer is None else layer
        t.tid = tid
        t.ctr = 0
        steps = C.c_uint64()
        nsec = C.c_uint64()
        path, edep, esc = C.c_double(), C.c_double(), C.c_double()
        status = lib().om_transport_track(self._h, event, C.byref(t), max_steps, C.byref(steps),
                                          C.byref(path), C.byref(edep), C.byref(esc), C.byref(nsec))
        return dict(status=status, steps=steps.value, path=path.value, edep=edep.value, escaped=esc.value,
                    secondaries=nsec.value, E=t.E, pos=(t.x, t.y, t.z), dir=(t.ux, t.uy, t.uz), layer=t.layer)


def primary_track_ids(events):
    """Track id of each primary: its running index within its event."""
    events = np.asarray(events)
    tids = np.zeros(len(events), dtype=np.uint64)
    counts = {}
    for i, e in enumerate(events.tolist()):
        c = counts.get(e, 0)
        tids[i] = c
        counts[e] = c + 1
    return tids


def philox(ctr, key):
    L = lib()
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    L.om_philox4x32_10(c, k, o)
    return list(o)


def raw_word(seed, event, tid, index):
    return lib().om_raw_word(seed, event, tid, index)


def uniform(w):
    return lib().om_uniform(w)


def rng(seed=1, event=0, tid=0, ctr=0):
    return om_rng(seed, event, tid, ctr)


def sigma_kn(E):
    return lib().om_sigma_kn(float(E))


def sigma_moller(T, Tcut):
    return lib().om_sigma_moller(float(T), float(Tcut))


def dedx_collision(T, Tcut, ne, I):
    return lib().om_dedx_collision(float(T), float(Tcut), float(ne), float(I))


def electron_density(m):
    mm = om_material(m.Z, m.A, m.rho, m.ne, m.X0, m.I)
    return lib().om_electron_density(C.byref(mm))


def gauss_legendre(n):
    x, w = np.zeros(n), np.zeros(n)
    lib().om_gauss_legendre(n, _arr(x), _arr(w))
    return x, w


def sample_compton(E, n, seed=7, event=0):
    eps, cost = np.zeros(n), np.zeros(n)
    e, c = C.c_double(), C.c_double()
    L = lib()
    for i in range(n):
        r = om_rng(seed, event, i, 0)
        L.om_sample_compton(float(E), C.byref(r), C.byref(e), C.byref(c))
        eps[i], cost[i] = e.value, c.value
    return eps, cost


def sample_moller(T, Tcut, n, seed=7):
    L = lib()
    out = np.zeros(n)
    for i in range(n):
        r = om_rng(seed, 0, i, 0)
        out[i] = L.om_sample_moller(float(T), float(Tcut), C.byref(r))
    return out


def sample_brems(T, kcut, n, seed=7):
    L = lib()
    out = np.zeros(n)
    for i in range(n):
        r = om_rng(seed, 0, i, 0)
        out[i] = L.om_sample_brems(float(T), float(kcut), C.byref(r))
    return out


def sample_isotropic(n, seed=7):
    L = lib()
    out = np.zeros((n, 3))
    d = (C.c_double * 3)()
    for i in range(n):
        r = om_rng(seed, 0, i, 0)
        L.om_sample_isotropic(C.byref(r), d)
        out[i] = list(d)
    return out


def rotate(u, cost, phi):
    uu = (C.c_double * 3)(*u)
    o = (C.c_double * 3)()
    lib().om_rotate(uu, float(cost), float(phi), o)
    return np.array(list(o))


def curvature(ptype, E, Bz):
    return lib().om_curvature(int(ptype), float(E), float(Bz))


def helix_move(kappa, s, pos, direction):
    p = (C.c_double * 3)(*pos)
    d = (C.c_double * 3)(*direction)
    lib().om_helix_move(float(kappa), float(s), p, d)
    return np.array(list(p)), np.array(list(d))


def rk_substeps(kappa, s):
    return lib().om_rk_substeps(float(kappa), float(s))


def rk_move(kappa, s, n, pos, direction):
    p = (C.c_double * 3)(*pos)
    d = (C.c_double * 3)(*direction)
    lib().om_rk_move(float(kappa), float(s), int(n), p, d)
    return np.array(list(p)), np.array(list(d))


def helix_side_distance(kappa, pos, direction, hx, hy):
    p = (C.c_double * 3)(*pos)
    d = (C.c_double * 3)(*direction)
    hit = C.c_int()
    s = lib().om_helix_side_distance(float(kappa), p, d, float(hx), float(hy), C.byref(hit))
    return s, hit.value
