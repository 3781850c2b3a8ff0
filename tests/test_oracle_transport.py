"""Pins of the oracle's transport loop (CPU only): closed-form laws the
stepping must reproduce, exact energy conservation, and scheduling
independence."""
import math

import numpy as np
import pytest

import oracle
from paper_2503_17608_gb300 import workloads as wl


def slab_problem(thickness, material, processes, **kw):
    base = dict(materials=[material], layer_material=[0], layer_thickness=[thickness], n_periods=1,
                half_x=1e6, half_y=1e6, Bz=0.0, cut_track=0.01, cut_moller=1.0, cut_brems=1.0,
                processes=processes, tally_mode=wl.TALLY_LAYERS, n_zbins=0, n_slots=1024, init_capacity=4096)
    base.update(kw)
    return wl.Problem(**base)


@pytest.mark.parametrize("E", [0.1, 1.0, 10.0])
def test_uncollided_transmission(E):
    """Fraction of photons crossing 10 cm of water without interacting is
    exp(-mu(E) * 10), mu from the oracle's own table lookup."""
    w = oracle.World(slab_problem(10.0, wl.WATER, wl.PHOTON_PROCS))
    n = 100000
    prim = wl.make_primaries(np.full(n, E), np.zeros((n, 3)), np.tile([0, 0, 1.0], (n, 1)),
                             np.zeros(n, np.int32), np.zeros(n, np.uint32))
    hist, _ = w.run(prim, with_edep=False)
    uncollided = (hist["steps"] == 1) & (hist["escaped"] == E)
    mu = sum(w.lookup(0, c, E) for c in (oracle.COL_COMPTON, oracle.COL_PE, oracle.COL_PAIR))
    p = math.exp(-mu * 10.0)
    sigma = math.sqrt(p * (1 - p) / n)
    assert abs(uncollided.mean() - p) < 4 * sigma


def check_conservation(prob, prim, rel=1e-12):
    w = oracle.World(prob)
    hist, edep = w.run(prim)
    per_primary = edep.sum(1) + hist["escaped"]
    np.testing.assert_allclose(per_primary, prim["E"], rtol=rel)
    for ev in np.unique(prim["event"]):
        m = prim["event"] == ev
        tot = edep[m].sum() + hist["escaped"][m].sum()
        assert tot == pytest.approx(prim["E"][m].sum(), rel=rel)
    return hist, edep


def test_energy_conservation_water_cube():
    hist, edep = check_conservation(wl.water_cube_problem(), wl.water_cube_primaries())
    assert hist["steps"].sum() > 20000
    # only pair production makes secondaries (two 511 keV photons)
    assert np.all(hist["secondaries"] % 2 == 0)


def test_energy_conservation_calorimeter():
    prob, prim = wl.calorimeter_1gev(40)
    hist, edep = check_conservation(prob, prim)
    assert np.all(hist["secondaries"] > 0)


def test_energy_conservation_field():
    prob, prim = wl.calorimeter_field_10gev(6)
    check_conservation(prob, prim)


def test_energy_conservation_event_mix():
    events = wl.offload_events(4)
    prim = wl.concat_primaries(events)[:600]
    prob = wl.calorimeter_problem(65536, Bz=4.0, max_events=4)
    check_conservation(prob, prim)


def test_oracle_results_do_not_depend_on_threads():
    prob, prim = wl.calorimeter_1gev(64)
    w = oracle.World(prob)
    h1, e1 = w.run(prim, n_threads=1)
    h8, e8 = w.run(prim, n_threads=8)
    np.testing.assert_array_equal(h1, h8)
    np.testing.assert_array_equal(e1, e8)


def test_brems_only_mean_energy_law():
    """Discrete 1/k brems only (no continuous loss): between emissions T is
    constant, so the mean energy after depth x obeys
    d<T>/dx = -(<T> - k_cut)/X0, i.e. <T(x)> = k_cut + (T0 - k_cut) e^{-x/X0}
    (up to the tiny probability of falling below k_cut)."""
    X0, T0, kcut = 0.56, 1000.0, 1.0
    mat = wl.Material("Pb-like", Z=82, A=207.2, rho=11.35, ne=0.0, X0=X0, I=823e-6)
    for x_over in (0.5, 1.0, 2.0):
        w = oracle.World(slab_problem(x_over * X0, mat, wl.PROC_BREMS, cut_track=1e-3))
        n = 20000
        Ts = np.empty(n)
        n_killed = 0
        for i in range(n):
            r = w.transport_track(T0, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), wl.ELECTRON, tid=i)
            # leaves through the back face, unless a photon took (almost) all of T
            assert r["status"] in (0, 1)
            Ts[i] = r["E"]
            assert r["dir"] == (0.0, 0.0, 1.0)
            n_killed += r["status"] == 0
        assert n_killed < 0.01 * n
        expect = kcut + (T0 - kcut) * math.exp(-x_over)
        assert abs(Ts.mean() - expect) < 4 * Ts.std() / math.sqrt(n) + 1e-3 * expect


def test_csda_path_matches_range_table():
    """Continuous loss only: the path travelled until the energy drops below the
    tracking cut equals R(E0) - R(E_final) from the range table."""
    prob = slab_problem(1e4, wl.LAR, wl.PROC_ELOSS, cut_track=0.1)
    w = oracle.World(prob)
    for E0 in (0.5, 3.0, 40.0, 900.0):
        r = w.transport_track(E0, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), wl.ELECTRON)
        assert r["status"] == 0
        Ef = r["E"]
        assert Ef < 0.1
        R0 = w.lookup(0, oracle.COL_RANGE, E0)
        Rf = w.lookup(0, oracle.COL_RANGE, Ef) if Ef > 1e-3 else 0.0
        if Ef > 1e-3:
            assert r["path"] == pytest.approx(R0 - Rf, rel=1e-9)
        else:
            assert R0 - w.table(0, oracle.COL_RANGE)[0] <= r["path"] <= R0 * (1 + 1e-12)
        assert r["edep"] == pytest.approx(E0, rel=1e-13)
        # range-limited steps shrink geometrically: 0.2 R per step above 0.1 cm
        assert r["steps"] >= 1


def test_escape_and_boundary_bookkeeping():
    """A photon with all processes off crosses every layer without interacting
    and escapes with its full energy after one step per layer."""
    prob = wl.calorimeter_problem(processes=0)
    w = oracle.World(prob)
    r = w.transport_track(5.0, (1.0, 2.0, 0.0), (0.0, 0.0, 1.0), wl.GAMMA)
    assert r["status"] == 1
    assert r["steps"] == prob.n_layers_total
    assert r["escaped"] == 5.0
    assert r["path"] == pytest.approx(28.0, rel=1e-12)
    # oblique photon leaves through a side plane
    d = np.array([0.9, 0.0, math.sqrt(1 - 0.81)])
    r = w.transport_track(5.0, (0.0, 0.0, 0.0), tuple(d), wl.GAMMA)
    assert r["status"] == 1
    assert r["pos"][0] == pytest.approx(50.0, rel=1e-12)


def test_tally_bins_water_cube():
    prob = wl.water_cube_problem()
    w = oracle.World(prob)
    prim = wl.water_cube_primaries(300)
    hist, edep = w.run(prim)
    assert edep.shape == (300, 100)
    prof = edep.sum(0)
    # 10 MeV photons along +z deposit mostly downstream of the entry face
    assert prof[:50].sum() > prof[50:].sum() > 0


def test_field_substep_cap_splits_steps_and_conserves_energy():
    """Runge-Kutta field propagation with a cap on the substeps of one step
    (Sec. 3.3): a cap cuts long curved steps into several, so the step count
    grows as the cap shrinks, while the shower's energy stays conserved and
    without a binding cap the substeps reproduce the exact helix's step count
    closely."""
    prob, prim = wl.calorimeter_field_10gev(6)
    hist_exact, edep_exact = oracle.World(prob).run(prim)
    steps = {}
    for cap in (1 << 30, 50, 3):
        p = prob.replace(field_substep_cap=cap)
        hist, edep = oracle.World(p).run(prim)
        total = edep.sum() + hist["escaped"].sum()
        assert total == pytest.approx(prim["E"].sum(), rel=1e-12)
        steps[cap] = int(hist["steps"].sum())
    exact = int(hist_exact["steps"].sum())
    assert abs(steps[1 << 30] - exact) < 0.01 * exact
    assert steps[1 << 30] <= steps[50] < steps[3]


def _first_steps(w, E0, n):
    """Path length of each of the first n steps of a continuous-loss-only
    electron (one thick layer, no discrete process: every step is range
    limited), from cumulative one-step-at-a-time runs."""
    paths, prev = [], 0.0
    for k in range(1, n + 1):
        r = w.transport_track(E0, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), wl.ELECTRON, max_steps=k)
        if r["steps"] < k:
            break
        paths.append(r["path"] - prev)
        prev = r["path"]
    return paths, r


def test_range_step_function_properties():
    """The range step limit (alpha_r = 0.2, f_r = 0.1 cm) is fixed by properties
    that any swap or misreading breaks:

    * at or below f_r the whole residual range is one step (s = R);
    * s is continuous at R = f_r (both sides give f_r);
    * s / R -> alpha_r = 0.2 as R grows (R = 3009 cm at 10 GeV in LAr);
    * a 1 MeV electron in LAr (R0 = 0.42431 cm, R(0.1 MeV) = 0.01473 cm) takes
      exactly 3 steps. By hand: s1 = 0.2 R0 + 0.08 (2 - 0.1 / R0)
      = 0.08486 + 0.14115 = 0.22601, R1 = 0.19830; s2 = 0.03966 + 0.11966
      = 0.15932, R2 = 0.03898 <= 0.1; s3 = R2 and the track stops. With
      alpha and f_r swapped it would take 2 steps (s1 = 0.31759, R1 = 0.10672 <= 0.2).
    """
    w = oracle.World(slab_problem(1e5, wl.LAR, wl.PROC_ELOSS, cut_track=0.1))
    R = lambda E: w.lookup(0, oracle.COL_RANGE, E)  # noqa: E731
    # s = R at and below f_r: one step ranges the electron out
    for E0 in (0.15, 0.3):
        assert R(E0) < 0.1
        r = w.transport_track(E0, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), wl.ELECTRON)
        assert r["steps"] == 1 and r["status"] == 0
        assert r["path"] == pytest.approx(R(E0), rel=1e-12)
    # continuity at f_r: energies whose range brackets 0.1 cm step by ~0.1 cm
    from scipy.optimize import brentq
    E_f = brentq(lambda E: R(E) - 0.1, 0.2, 1.0, xtol=1e-15)
    for dE in (-1e-6, 1e-6):
        paths, _ = _first_steps(w, E_f + dE, 1)
        assert paths[0] == pytest.approx(0.1, abs=1e-5)
    # s / R -> 0.2 for a long residual range
    paths, _ = _first_steps(w, 1e4, 1)
    assert R(1e4) > 1000.0
    assert abs(paths[0] / R(1e4) - 0.2) < 1e-4
    # the hand-derived sequence at 1 MeV
    paths, r = _first_steps(w, 1.0, 5)
    assert len(paths) == 3 and r["status"] == 0
    np.testing.assert_allclose(paths[:2], [0.22601, 0.15932], atol=2e-5)
    assert sum(paths) == pytest.approx(R(1.0), rel=1e-12)
    # every range-limited step is shorter than the residual range
    paths, _ = _first_steps(w, 50.0, 8)
    Rk = R(50.0)
    for s in paths:
        assert 0.2 * Rk < s < Rk
        Rk -= s
