"""The CPU oracle against the fixtures in tests/golden/: published reference
values (each with its source in reference_values.txt) and a regression record
of water-cube histories written by tests/golden/make_water_cube_histories.py
from the oracle itself (a change to the oracle's arithmetic shows up here)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2503_17608_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def reference_values():
    out = {}
    with open(os.path.join(GOLDEN, "reference_values.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            name, value, unit, tol, source = [x.strip() for x in line.split("|", 4)]
            out[name] = (float(value), float(tol), source)
    return out


REF = reference_values()


def test_every_reference_value_has_a_source():
    assert len(REF) >= 7
    for name, (_, _, source) in REF.items():
        assert len(source) > 20, name


def test_klein_nishina_at_one_mev():
    v, tol, _ = REF["kn_sigma_1mev"]
    assert oracle.sigma_kn(1.0) == pytest.approx(v, rel=tol)


def thomson_from_oracle():
    """sigma_T from the oracle's closed form at 1 keV (the low end of its
    tables, where the cancellation in the closed form costs ~1e-11) divided by
    the Thomson-limit series 1 - 2k + 26/5 k^2 - 133/10 k^3 + 1144/35 k^4."""
    me = REF["electron_mass"][0]
    k = 1e-3 / me
    series = 1.0 - 2.0 * k + 26.0 / 5.0 * k**2 - 133.0 / 10.0 * k**3 + 1144.0 / 35.0 * k**4
    return oracle.sigma_kn(1e-3) / series


def test_thomson_limit():
    v, tol, _ = REF["thomson_sigma"]
    assert thomson_from_oracle() == pytest.approx(v, rel=tol)


def test_electron_mass_and_radius():
    # the oracle's electron mass, recovered from its curvature: |kappa| = c B / p, p^2 = E^2 + 2 m E
    me, tol, _ = REF["electron_mass"]
    E, B = 3.0, 2.0
    p = 2.99792458 * B / abs(oracle.curvature(wl.ELECTRON, E, B))
    assert (p * p - E * E) / (2.0 * E) == pytest.approx(me, rel=tol)
    # its classical radius, from the Thomson limit 8 pi r_e^2 / 3
    re, tol_r, _ = REF["classical_radius"]
    assert math.sqrt(3.0 * thomson_from_oracle() / (8.0 * math.pi)) == pytest.approx(re, rel=1e-8)


def test_water_cube_coefficients():
    w = oracle.World(wl.water_cube_problem())
    lnE = w.grid()
    E = np.exp(lnE)
    v, tol, _ = REF["water_pe_30kev"]
    np.testing.assert_allclose(w.table(0, oracle.COL_PE), v * (E / 0.030) ** -3.5, rtol=tol)
    slope, tol2, _ = REF["water_pair_10mev"]
    above = E > 1.022
    np.testing.assert_allclose(w.table(0, oracle.COL_PAIR)[above], slope * np.log(E[above] / 1.022), rtol=tol2)


def test_water_stopping_power():
    v, tol, _ = REF["water_stopping_1mev"]
    S = oracle.dedx_collision(1.0, 1e9, 3.343e23, 75e-6)
    assert v <= S <= v * (1.0 + tol)


def test_water_cube_histories_regression():
    rows = np.loadtxt(os.path.join(GOLDEN, "water_cube_histories.txt"))
    n = len(rows)
    hist, edep = oracle.World(wl.water_cube_problem()).run(wl.water_cube_primaries(n), n_threads=2)
    np.testing.assert_array_equal(hist["steps"], rows[:, 1].astype(np.uint64))
    np.testing.assert_array_equal(hist["secondaries"], rows[:, 2].astype(np.uint64))
    np.testing.assert_allclose(edep.sum(axis=1), rows[:, 3], rtol=1e-15, atol=1e-13)
    np.testing.assert_allclose(hist["escaped"], rows[:, 4], rtol=1e-15, atol=1e-13)
