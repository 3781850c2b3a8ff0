"""Seeded synthetic workloads: problem descriptions and primary particles.

This module is the only code shared by the CUDA path and the CPU oracle. It
holds plain data (materials, layer stacks, cuts, slot counts) and seeded
random draws of primary particles; it contains none of the transport
arithmetic (no cross sections, no stepping, no random streams of the method).

The paper benchmarks on detector geometries with 10 GeV electron showers
(Sec. 5: 16 events x 1300 primaries, uniform 1 T / 3.8 T fields). Those
geometries are not available, so the layered sampling calorimeters below stand
in for them: lead/liquid-argon slabs (shape of a sampling calorimeter such as
TestEM3), a uniform field along z, and 1-10 GeV electron primaries.

Units: MeV, cm, tesla, g/cm3.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

# Particle types (the track-state "particle type" field, Sec. 2).
GAMMA = 0
ELECTRON = 1
POSITRON = 2

# Process bitmask.
PROC_COMPTON = 1
PROC_PHOTOELECTRIC = 2
PROC_PAIR = 4
PROC_MOLLER = 8
PROC_BREMS = 16
PROC_ELOSS = 32
PHOTON_PROCS = PROC_COMPTON | PROC_PHOTOELECTRIC | PROC_PAIR
ALL_PROCS = PHOTON_PROCS | PROC_MOLLER | PROC_BREMS | PROC_ELOSS

# Tally layouts.
TALLY_ZBINS = 0
TALLY_LAYERS = 1

# Track-reordering policies (Sec. 3.1).
SORT_NONE = 0
SORT_ACTION = 1
SORT_ACTION_TYPE = 2
SORT_LOCAL = 3
SORT_DATA = 4
SORT_NAMES = {"none": SORT_NONE, "action": SORT_ACTION, "action_type": SORT_ACTION_TYPE, "local": SORT_LOCAL,
              "data": SORT_DATA}

DEFAULT_SEED = 20250321

# Primary record dtype (host side, array of structs).
PRIMARY_DTYPE = np.dtype(
    [
        ("E", np.float64),
        ("pos", np.float64, (3,)),
        ("dir", np.float64, (3,)),
        ("ptype", np.int32),
        ("event", np.uint32),
    ]
)


@dataclasses.dataclass
class Material:
    name: str
    Z: float          # atomic number (effective Z for a compound)
    A: float          # g/mol (0 when ne is given directly)
    rho: float        # g/cm3
    ne: float         # electrons/cm3; 0 means "derive from N_A rho Z / A"
    X0: float         # radiation length, cm
    I: float          # mean excitation energy, MeV


WATER = Material("water", Z=7.42, A=0.0, rho=1.0, ne=3.343e23, X0=36.08, I=78.0e-6)
LEAD = Material("Pb", Z=82.0, A=207.2, rho=11.35, ne=0.0, X0=0.56, I=823.0e-6)
LAR = Material("LAr", Z=18.0, A=39.948, rho=1.39, ne=0.0, X0=14.0, I=188.0e-6)


@dataclasses.dataclass
class Problem:
    materials: List[Material]
    layer_material: List[int]
    layer_thickness: List[float]
    n_periods: int
    half_x: float
    half_y: float
    Bz: float
    cut_track: float
    cut_moller: float
    cut_brems: float
    processes: int
    tally_mode: int
    n_zbins: int
    n_slots: int
    init_capacity: int
    max_events: int = 1
    history_capacity: int = 0
    sort_policy: int = SORT_NONE
    block_size: int = 256
    split_actions: int = 0
    seed: int = DEFAULT_SEED
    field_substep_cap: int = 0  # 0: exact helix; > 0: Runge-Kutta substeps, at most this many per step
    name: str = ""

    @property
    def n_layers_total(self) -> int:
        return len(self.layer_material) * self.n_periods

    @property
    def n_bins(self) -> int:
        return self.n_layers_total if self.tally_mode == TALLY_LAYERS else self.n_zbins

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def make_primaries(E, pos, direction, ptype, event) -> np.ndarray:
    n = len(E)
    p = np.zeros(n, dtype=PRIMARY_DTYPE)
    p["E"] = E
    p["pos"] = pos
    p["dir"] = direction
    p["ptype"] = ptype
    p["event"] = event
    return p


# --------------------------------------------------------------------------
# Photon-only water cube (2,000 x 10 MeV photons, 4,096 slots).
# --------------------------------------------------------------------------
def water_cube_problem(n_slots: int = 4096, **kw) -> Problem:
    base = dict(
        materials=[WATER],
        layer_material=[0],
        layer_thickness=[100.0],
        n_periods=1,
        half_x=50.0,
        half_y=50.0,
        Bz=0.0,
        cut_track=0.010,
        cut_moller=1.0,
        cut_brems=1.0,
        processes=PHOTON_PROCS,
        tally_mode=TALLY_ZBINS,
        n_zbins=100,
        n_slots=n_slots,
        init_capacity=4 * n_slots,
        name="water-cube photons 10 MeV",
    )
    base.update(kw)
    return Problem(**base)


def water_cube_primaries(n: int = 2000, energy: float = 10.0, event: int = 0) -> np.ndarray:
    return make_primaries(
        np.full(n, energy),
        np.zeros((n, 3)),
        np.tile([0.0, 0.0, 1.0], (n, 1)),
        np.full(n, GAMMA, np.int32),
        np.full(n, event, np.uint32),
    )


# --------------------------------------------------------------------------
# Lead/liquid-argon sampling calorimeter: 40 x (2 mm Pb + 5 mm LAr), 1 m x 1 m.
# --------------------------------------------------------------------------
def calorimeter_problem(n_slots: int = 65536, Bz: float = 0.0, **kw) -> Problem:
    base = dict(
        materials=[LEAD, LAR],
        layer_material=[0, 1],
        layer_thickness=[0.2, 0.5],
        n_periods=40,
        half_x=50.0,
        half_y=50.0,
        Bz=Bz,
        cut_track=0.100,
        cut_moller=1.0,
        cut_brems=1.0,
        processes=ALL_PROCS,
        tally_mode=TALLY_LAYERS,
        n_zbins=0,
        n_slots=n_slots,
        init_capacity=8 * n_slots,
        name="Pb/LAr calorimeter" + (f" Bz={Bz} T" if Bz else ""),
    )
    base.update(kw)
    return Problem(**base)


def electron_beam(n: int, energy: float, event: int = 0, patch_half: float = 0.0,
                  seed: int = DEFAULT_SEED) -> np.ndarray:
    """Electrons along +z starting on the front face (z = 0); start points uniform
    over a square patch of half-width ``patch_half`` (0: all at the origin)."""
    pos = np.zeros((n, 3))
    if patch_half > 0:
        rng = np.random.default_rng(seed)
        pos[:, 0:2] = rng.uniform(-patch_half, patch_half, size=(n, 2))
    return make_primaries(
        np.full(n, energy), pos, np.tile([0.0, 0.0, 1.0], (n, 1)),
        np.full(n, ELECTRON, np.int32), np.full(n, event, np.uint32),
    )


def calorimeter_1gev(n: int = 1000) -> tuple[Problem, np.ndarray]:
    """1,000 x 1 GeV electrons, no field, 65,536 slots."""
    return calorimeter_problem(65536), electron_beam(n, 1000.0)


def calorimeter_field_10gev(n: int = 10000, n_slots: int = 1 << 20) -> tuple[Problem, np.ndarray]:
    """10,000 x 10 GeV electrons in a 4 T field along z, start points uniform over
    a 10 cm x 10 cm patch of the front face, 2^20 slots."""
    prob = calorimeter_problem(n_slots, Bz=4.0)
    return prob, electron_beam(n, 10000.0, patch_half=5.0)


# --------------------------------------------------------------------------
# Offload-style event mix: lognormal event sizes (median 200, sigma 1), 50/50
# photons/electrons, energies log-uniform in [100 MeV, 10 GeV], start points
# uniform over the front face.
# --------------------------------------------------------------------------
def offload_event(rng: np.random.Generator, event: int, half: float = 50.0) -> np.ndarray:
    n = int(math.ceil(rng.lognormal(mean=math.log(200.0), sigma=1.0)))
    n = max(n, 1)
    E = np.exp(rng.uniform(math.log(100.0), math.log(10000.0), size=n))
    pos = np.zeros((n, 3))
    pos[:, 0:2] = rng.uniform(-half, half, size=(n, 2))
    ptype = np.where(rng.uniform(size=n) < 0.5, GAMMA, ELECTRON).astype(np.int32)
    return make_primaries(E, pos, np.tile([0.0, 0.0, 1.0], (n, 1)), ptype,
                          np.full(n, event, np.uint32))


def offload_events(n_events: int = 256, seed: int = DEFAULT_SEED, first_event: int = 0) -> List[np.ndarray]:
    rng = np.random.default_rng([seed, 0xFFFFFFFF])
    return [offload_event(rng, first_event + i) for i in range(n_events)]


def poisson_arrivals(rate_hz: float = 2000.0, duration_s: float = 60.0,
                     seed: int = DEFAULT_SEED) -> np.ndarray:
    """Arrival times (s) of a Poisson process."""
    rng = np.random.default_rng([seed, 0xFFFFFFFE])
    n_expect = int(rate_hz * duration_s * 1.2) + 100
    gaps = rng.exponential(1.0 / rate_hz, size=n_expect)
    t = np.cumsum(gaps)
    return t[t < duration_s]


def concat_primaries(events: Sequence[np.ndarray]) -> np.ndarray:
    return np.concatenate(list(events)) if events else np.zeros(0, PRIMARY_DTYPE)
