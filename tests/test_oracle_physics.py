"""Pins of the oracle's physics definitions (CPU only).

Each check compares the oracle against something other than itself: a
differential cross-section integrated numerically, a textbook anchor value,
an algebraic identity between two independently written formulas, a library
routine, or a closed-form law of the sampled distribution.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle
from paper_2503_17608_gb300 import workloads as wl

ME = 0.51099895
RE = 2.8179403262e-13


# ---------------------------------------------------------------- Compton
def kn_dsigma_dcos(E, c):
    """Klein-Nishina differential cross-section per electron, d sigma / d cos(theta)."""
    k = E / ME
    P = 1.0 / (1.0 + k * (1.0 - c))
    return np.pi * RE**2 * P * P * (P + 1.0 / P - (1.0 - c * c))


@pytest.mark.parametrize("E", [0.01, 0.1, 0.511, 1.0, 10.0, 100.0, 1e4])
def test_kn_total_equals_integral_of_differential(E):
    val, err = integrate.quad(lambda c: kn_dsigma_dcos(E, c), -1, 1, epsabs=0, epsrel=1e-13, limit=200)
    tol = 1e-9 if E >= 0.1 else 1e-7
    assert oracle.sigma_kn(E) == pytest.approx(val, rel=tol)


def test_kn_textbook_anchor_and_thomson_limit():
    # 1 MeV: 0.2112 barn per electron (Compton, free electron)
    assert oracle.sigma_kn(1.0) == pytest.approx(0.2112e-24, rel=2e-3)
    sigma_t = 8 * np.pi / 3 * RE**2
    k = 1e-3 / ME
    # low-energy expansion sigma / sigma_T = 1 - 2k + 26/5 k^2 - ...
    assert oracle.sigma_kn(1e-3) / sigma_t == pytest.approx(1 - 2 * k + 5.2 * k * k, abs=50 * k**3 + 1e-9)


def kn_cdf(E, n=40001):
    c = np.linspace(-1, 1, n)
    f = kn_dsigma_dcos(E, c)
    F = integrate.cumulative_trapezoid(f, c, initial=0.0)
    F /= F[-1]
    return lambda x: np.interp(x, c, F)


@pytest.mark.parametrize("E", [0.01, 0.511, 10.0])
def test_kn_angular_sampling_ks(E):
    eps, cost = oracle.sample_compton(E, 100000, seed=11)
    assert np.all((cost >= -1) & (cost <= 1))
    # energy and angle are tied by Compton kinematics
    k = E / ME
    np.testing.assert_allclose(eps, 1.0 / (1.0 + k * (1.0 - cost)), rtol=1e-12)
    assert stats.kstest(cost, kn_cdf(E)).pvalue > 1e-3


def test_kn_sampling_thomson_limit():
    # at 1 keV the angular law is the Thomson one, (1 + cos^2) / (8/3)
    _, cost = oracle.sample_compton(1e-3, 100000, seed=5)
    cdf = lambda c: (c + c**3 / 3 + 4 / 3) / (8 / 3)
    assert stats.kstest(cost, cdf).pvalue > 1e-3


# ---------------------------------------------------------------- tables
def test_config_anchor_values():
    w = oracle.World(wl.water_cube_problem())
    # photoelectric: 0.15 / cm at 30 keV (interpolation linear in ln E)
    assert w.lookup(0, oracle.COL_PE, 0.030) == pytest.approx(0.15, rel=0.02)
    # pair: 0.0096 / cm ln(E / 1.022 MeV)
    E = 1.022 * math.e**2
    assert w.lookup(0, oracle.COL_PAIR, E) == pytest.approx(2 * 0.0096, rel=1e-3)
    # Compton = n_e sigma_KN
    assert w.lookup(0, oracle.COL_COMPTON, 1.0) == pytest.approx(3.343e23 * 0.2112e-24, rel=3e-3)
    # water: Z/Z_w = 1 and n_e = n_e,w, so no scaling
    lnE = w.grid()
    np.testing.assert_allclose(w.table(0, oracle.COL_PE), 0.15 * (np.exp(lnE) / 0.03) ** -3.5, rtol=1e-12)


def test_z_scaling_of_photon_processes():
    w = oracle.World(wl.calorimeter_problem())
    ww = oracle.World(wl.water_cube_problem())
    ne_pb = oracle.electron_density(wl.LEAD)
    assert ne_pb == pytest.approx(6.02214076e23 * 11.35 * 82 / 207.2, rel=1e-15)
    r = ne_pb / 3.343e23
    z = 82 / 7.42
    np.testing.assert_allclose(w.table(0, oracle.COL_PE), r * z**3 * ww.table(0, oracle.COL_PE), rtol=1e-12)
    np.testing.assert_allclose(w.table(0, oracle.COL_PAIR), r * z * ww.table(0, oracle.COL_PAIR), rtol=1e-12)
    np.testing.assert_allclose(w.table(0, oracle.COL_COMPTON), r * ww.table(0, oracle.COL_COMPTON), rtol=1e-12)


def test_pair_threshold_is_hard():
    w = oracle.World(wl.water_cube_problem())
    # below threshold the photon never pair-produces, whatever the interpolation gives
    for E in (1.0, 1.02, 1.0219, 1.022):
        for u in np.linspace(0.001, 0.999, 51):
            assert w.select_process(0, wl.GAMMA, E, u) != oracle.SEL_PAIR


def test_process_selection_frequencies():
    w = oracle.World(wl.calorimeter_problem())
    for mat, ptype, E, cols in ((0, wl.GAMMA, 5.0, (0, 1, 2)), (1, wl.GAMMA, 0.2, (0, 1, 2)),
                                (0, wl.ELECTRON, 50.0, (3, 4)), (1, wl.ELECTRON, 500.0, (3, 4))):
        n = 20000
        u = (np.arange(n) + 0.5) / n
        sel = np.array([w.select_process(mat, ptype, E, x) for x in u])
        mu = np.array([w.lookup(mat, c, E) for c in cols])
        frac = np.array([(sel == (c if ptype == wl.GAMMA else c)).mean() for c in cols])
        np.testing.assert_allclose(frac, mu / mu.sum(), atol=2.0 / n)


# ---------------------------------------------------------------- charged
def moller_dsigma_deps(T, eps):
    """Moller differential cross-section per target electron, d sigma / d eps."""
    g = T / ME + 1
    b2 = 1 - 1 / g**2
    B = ((g - 1) ** 2 / g**2 + 1 / eps**2 - (2 * g - 1) / (g**2 * eps)
         + 1 / (1 - eps) ** 2 - (2 * g - 1) / (g**2 * (1 - eps)))
    return 2 * np.pi * RE**2 / (b2 * (g - 1)) * B


@pytest.mark.parametrize("T", [2.5, 10.0, 1000.0, 1e4])
def test_moller_total_equals_integral(T):
    Tcut = 1.0
    x = Tcut / T
    val, _ = integrate.quad(lambda e: moller_dsigma_deps(T, e), x, 0.5, epsabs=0, epsrel=1e-13, limit=200)
    assert oracle.sigma_moller(T, Tcut) == pytest.approx(val, rel=1e-10)
    assert oracle.sigma_moller(1.99, 1.0) == 0.0


@pytest.mark.parametrize("T", [3.0, 50.0, 5000.0])
def test_moller_sampling_chi2(T):
    Tcut = 1.0
    x = Tcut / T
    eps = oracle.sample_moller(T, Tcut, 60000, seed=3)
    assert np.all((eps >= x) & (eps <= 0.5))
    edges = x / (1 - np.linspace(0, 1, 41) * (1 - 2 * x))  # equal-probability bins of the proposal
    counts, _ = np.histogram(eps, edges)
    p = np.array([integrate.quad(lambda e: moller_dsigma_deps(T, e), a, b, epsrel=1e-12)[0]
                  for a, b in zip(edges[:-1], edges[1:])])
    p /= p.sum()
    chi2 = ((counts - len(eps) * p) ** 2 / (len(eps) * p)).sum()
    assert stats.chi2.sf(chi2, len(p) - 1) > 1e-3


def test_moller_rejection_bound():
    # the acceptance function never exceeds 1 on [x, 1/2]
    for T in (2.01, 3.0, 10.0, 1e3, 1e4):
        g = T / ME + 1
        eps = np.linspace(1.0 / T, 0.5, 10001)
        om = 1 - eps
        f = (g - 1) ** 2 * eps**2 - (2 * g * g + 2 * g - 1) * eps / om + g * g / om**2
        assert np.max(4 / (9 * g * g - 10 * g + 5) * f) <= 1 + 1e-12


def unrestricted_icru37(T, ne, I):
    """Electron collision stopping power, unrestricted, in the ICRU-37 form."""
    tau = T / ME
    g = tau + 1
    b2 = tau * (tau + 2) / g**2
    F = 1 - b2 + (tau**2 / 8 - (2 * tau + 1) * math.log(2)) / g**2
    return 2 * np.pi * RE**2 * ME * ne / b2 * (math.log(tau**2 * (tau + 2) / (2 * (I / ME) ** 2)) + F)


@pytest.mark.parametrize("T", [0.01, 0.3, 1.0, 1.9])
def test_restricted_dedx_reduces_to_unrestricted(T):
    # with the cut above T/2 the restricted formula is the full Bethe formula
    ne, I = oracle.electron_density(wl.LEAD), 823e-6
    assert oracle.dedx_collision(T, 1.0, ne, I) == pytest.approx(unrestricted_icru37(T, ne, I), rel=1e-12)


@pytest.mark.parametrize("T", [10.0, 300.0, 5000.0])
def test_restricted_dedx_derivative_is_moller_energy_loss(T):
    # S(W2) - S(W1) = ne * integral_{W1}^{W2} W d sigma/dW: the energy carried by
    # delta rays between the two cuts, from the Moller differential cross-section
    ne, I = oracle.electron_density(wl.LAR), 188e-6
    W1, W2 = 0.5, 2.0
    dS = oracle.dedx_collision(T, W2, ne, I) - oracle.dedx_collision(T, W1, ne, I)
    integral, _ = integrate.quad(lambda e: e * T * moller_dsigma_deps(T, e), W1 / T, W2 / T, epsrel=1e-12)
    assert dS == pytest.approx(ne * integral, rel=1e-9)


def test_water_stopping_power_anchor():
    # water, 1 MeV electrons, I = 75 eV: 1.849 MeV cm2/g with the density
    # effect; without it (as here) about 1.3% higher
    S = oracle.dedx_collision(1.0, 1e9, 3.343e23, 75e-6)
    assert 1.849 < S < 1.849 * 1.03


def test_gauss_legendre_matches_library():
    x, w = oracle.gauss_legendre(16)
    xl, wl_ = np.polynomial.legendre.leggauss(16)
    order = np.argsort(x)
    np.testing.assert_allclose(x[order], xl, atol=1e-15)
    np.testing.assert_allclose(w[order], wl_, rtol=1e-13)


def test_range_table_is_integral_of_inverse_stopping_power():
    prob = wl.calorimeter_problem()
    w = oracle.World(prob)
    lnE = w.grid()
    E = np.exp(lnE)
    for mat, m in enumerate(prob.materials):
        ne = oracle.electron_density(m)

        def S(e):
            return oracle.dedx_collision(e, prob.cut_moller, ne, m.I) + min(e, prob.cut_brems) / m.X0

        R = w.table(mat, oracle.COL_RANGE)
        dedx = w.table(mat, oracle.COL_DEDX)
        assert np.all(dedx > 0)
        assert R[0] == pytest.approx(E[0] / (2 * S(E[0])), rel=1e-14)
        for i in (1, 10, 57, 120, 199):
            val, _ = integrate.quad(lambda t: math.exp(t) / S(math.exp(t)), lnE[0], lnE[i], epsrel=1e-12,
                                    limit=400)
            # S has kinks at k_cut (radiative part) and 2 T_cut (restriction), where a
            # per-bin 16-point rule is only accurate to ~1e-8
            assert R[i] == pytest.approx(R[0] + val, rel=1e-7)
        assert np.all(np.diff(R) > 0)


def test_inverse_range_round_trip():
    w = oracle.World(wl.calorimeter_problem())
    rng = np.random.default_rng(4)
    for mat in (0, 1):
        for E in np.exp(rng.uniform(math.log(2e-3), math.log(9e3), 300)):
            r = w.lookup(mat, oracle.COL_RANGE, E)
            assert w.inv_range(mat, r) == pytest.approx(E, rel=1e-12)


def test_brems_spectrum_ks():
    T, kcut = 800.0, 1.0
    k = oracle.sample_brems(T, kcut, 50000, seed=9)
    assert np.all((k > kcut) & (k <= T))
    assert stats.kstest(k, lambda x: np.log(x / kcut) / np.log(T / kcut)).pvalue > 1e-3


# ---------------------------------------------------------------- kinematics
def test_isotropic_directions():
    d = oracle.sample_isotropic(60000, seed=2)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1, rtol=1e-14)
    assert stats.kstest(d[:, 2], "uniform", args=(-1, 2)).pvalue > 1e-3
    phi = np.arctan2(d[:, 1], d[:, 0])
    assert stats.kstest(phi, "uniform", args=(-np.pi, 2 * np.pi)).pvalue > 1e-3


def test_rotation_preserves_polar_angle():
    rng = np.random.default_rng(8)
    for _ in range(500):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        if rng.uniform() < 0.1:
            u = np.array([0.0, 0.0, rng.choice([-1.0, 1.0])])
        c, phi = rng.uniform(-1, 1), rng.uniform(0, 2 * np.pi)
        v = oracle.rotate(u, c, phi)
        assert np.linalg.norm(v) == pytest.approx(1, abs=1e-14)
        assert np.dot(u, v) == pytest.approx(c, abs=1e-12)
    # averaged over the azimuth, the rotated vector is cos(theta) u
    u = np.array([0.3, -0.4, np.sqrt(1 - 0.25)])
    vs = np.array([oracle.rotate(u, 0.2, p) for p in np.linspace(0, 2 * np.pi, 4096, endpoint=False)])
    np.testing.assert_allclose(vs.mean(0), 0.2 * u, atol=1e-12)


def lorentz_rhs(kappa):
    def f(s, y):
        ux, uy, uz = y[3:]
        return [ux, uy, uz, kappa * uy, -kappa * ux, 0.0]
    return f


def test_rotation_frame_is_the_written_convention():
    """The rotation frame (e1 = u x z / |u x z|, e2 = u x e1; along the z axis
    e1 = x, e2 = u x x / |u x x|) fixes where the azimuth phi = 0 and pi/2
    point: a reflected or rotated azimuth fails here.

    u = x: u x z = (0, -1, 0) = e1, e2 = x x (0, -1, 0) = (0, 0, -1).
    u = z: e1 = x, e2 = z x x = (0, 1, 0). u = -z: e2 = -z x x = (0, -1, 0).
    u = y: e1 = y x z = (1, 0, 0), e2 = y x x = (0, 0, -1).
    With cos(theta) = 0 the result is cos(phi) e1 + sin(phi) e2."""
    cases = [((1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (0.0, 0.0, -1.0)),
             ((0.0, 0.0, 1.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0)),
             ((0.0, 0.0, -1.0), (1.0, 0.0, 0.0), (0.0, -1.0, 0.0)),
             ((0.0, 1.0, 0.0), (1.0, 0.0, 0.0), (0.0, 0.0, -1.0))]
    for u, e1, e2 in cases:
        np.testing.assert_allclose(oracle.rotate(u, 0.0, 0.0), e1, atol=1e-15)
        np.testing.assert_allclose(oracle.rotate(u, 0.0, np.pi / 2), e2, atol=1e-15)
        np.testing.assert_allclose(oracle.rotate(u, 0.0, np.pi), -np.array(e1), atol=1e-15)
        # cos(theta) = 1 leaves the direction alone, -1 reverses it
        np.testing.assert_allclose(oracle.rotate(u, 1.0, 0.7), u, atol=1e-15)
        np.testing.assert_allclose(oracle.rotate(u, -1.0, 0.7), -np.array(u), atol=1e-15)
    # an oblique direction: e1 and e2 from the cross products, by hand
    u = np.array([0.36, 0.48, 0.8])
    n = np.hypot(u[0], u[1])
    e1 = np.array([u[1], -u[0], 0.0]) / n
    e2 = np.array([u[2] * u[0] / n, u[2] * u[1] / n, -n])
    c, phi = 0.3, 1.1
    want = c * u + np.sqrt(1 - c * c) * (np.cos(phi) * e1 + np.sin(phi) * e2)
    np.testing.assert_allclose(oracle.rotate(u, c, phi), want, atol=1e-15)


def test_helix_matches_equation_of_motion():
    from scipy.integrate import solve_ivp
    E, B = 7.0, 4.0
    kappa = oracle.curvature(wl.ELECTRON, E, B)
    p = math.sqrt(E * (E + 2 * ME))
    # |kappa| = c B / p with c = 2.99792458 [MeV / (T cm)]... radius p / (q B)
    assert abs(kappa) == pytest.approx(2.99792458 * B / p, rel=1e-15)
    assert kappa < 0
    u0 = np.array([0.6, 0.0, 0.8])
    x0 = np.array([1.0, -2.0, 3.0])
    for s in (0.01, 0.7, 3.3):
        pos, d = oracle.helix_move(kappa, s, x0, u0)
        sol = solve_ivp(lorentz_rhs(kappa), (0, s), list(x0) + list(u0), rtol=1e-12, atol=1e-13, method="DOP853")
        np.testing.assert_allclose(pos, sol.y[:3, -1], atol=1e-9)
        np.testing.assert_allclose(d, sol.y[3:, -1], atol=1e-9)


def test_helix_radius_and_period():
    E, B = 25.0, 4.0
    kappa = oracle.curvature(wl.ELECTRON, E, B)
    u = np.array([0.48, 0.6, 0.64])
    x0 = np.array([0.0, 0.0, 5.0])
    pperp = math.sqrt(E * (E + 2 * ME)) * math.hypot(u[0], u[1])
    rho = pperp / (2.99792458 * B)  # p_perp / (|q| B) in cm for MeV/c and T
    # centre from the helix itself: two points half a turn apart are a diameter apart
    period = 2 * math.pi / abs(kappa)
    p_half, _ = oracle.helix_move(kappa, period / 2, x0, u)
    assert math.hypot(*(p_half - x0)[:2]) == pytest.approx(2 * rho, rel=1e-12)
    p_full, d_full = oracle.helix_move(kappa, period, x0, u)
    assert np.linalg.norm((p_full - x0)[:2]) < 1e-10 * rho
    assert p_full[2] - x0[2] == pytest.approx(u[2] * period, rel=1e-14)
    np.testing.assert_allclose(d_full, u, atol=1e-12)


def test_helix_straight_limit_along_field():
    kappa = oracle.curvature(wl.ELECTRON, 10.0, 4.0)
    pos, d = oracle.helix_move(kappa, 2.5, [1.0, 2.0, 0.0], [0.0, 0.0, 1.0])
    np.testing.assert_array_equal(pos, [1.0, 2.0, 2.5])
    np.testing.assert_array_equal(d, [0.0, 0.0, 1.0])
    s, hit = oracle.helix_side_distance(kappa, [1.0, 2.0, 0.0], [0.0, 0.0, 1.0], 50, 50)
    assert s == math.inf and hit == 0


def test_helix_side_distance_brute_force():
    rng = np.random.default_rng(12)
    n_hit = 0
    for _ in range(60):
        E = float(np.exp(rng.uniform(np.log(5.0), np.log(2000.0))))
        kappa = oracle.curvature(wl.ELECTRON, E, 4.0)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        x0 = np.array([rng.uniform(-40, 40), rng.uniform(-40, 40), 1.0])
        hx = hy = 50.0
        s, hit = oracle.helix_side_distance(kappa, x0, u, hx, hy)
        # brute force: march along the helix and bisect the first exit
        period = 2 * math.pi / abs(kappa)
        ss = np.linspace(0, period, 20001)
        inside = []
        for t in ss:
            p, _ = oracle.helix_move(kappa, t, x0, u)
            inside.append(abs(p[0]) < hx and abs(p[1]) < hy)
        inside = np.array(inside)
        if inside.all():
            assert not hit
            continue
        n_hit += 1
        j = int(np.argmin(inside))
        a, b = ss[j - 1], ss[j]
        for _ in range(80):
            mid = 0.5 * (a + b)
            p, _ = oracle.helix_move(kappa, mid, x0, u)
            if abs(p[0]) < hx and abs(p[1]) < hy:
                a = mid
            else:
                b = mid
        assert hit
        assert s == pytest.approx(0.5 * (a + b), rel=1e-9, abs=1e-9)
    assert n_hit > 5


# ------------------------------------------------------------------ Runge-Kutta field substeps (Sec. 3.3)
def test_rk_substep_count():
    kappa = -2.5
    assert oracle.rk_substeps(kappa, 0.0) == 1
    assert oracle.rk_substeps(kappa, 0.04) == 1    # 0.1 rad of turn per substep at most
    assert oracle.rk_substeps(kappa, 0.041) == 2
    assert oracle.rk_substeps(kappa, 1.0) == 25
    assert oracle.rk_substeps(kappa, 1.0001) == 26


def test_rk_matches_equation_of_motion_within_fourth_order():
    """The Runge-Kutta path agrees with a DOP853 solution of the equation of
    motion to the classical fourth-order bound: per substep of turn angle
    theta the local error is ~theta^5 / 120 of the radius, so after n substeps
    of 0.1 rad at most ~1e-7 n rho; z advances by uz s exactly."""
    from scipy.integrate import solve_ivp
    rng = np.random.default_rng(21)
    for _ in range(20):
        E = float(np.exp(rng.uniform(np.log(1.0), np.log(500.0))))
        kappa = oracle.curvature(wl.ELECTRON, E, 4.0)
        rho = 1.0 / abs(kappa)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        x0 = rng.uniform(-5, 5, 3)
        s = float(rng.uniform(0.1, 30.0)) * rho
        n = oracle.rk_substeps(kappa, s)
        pos, d = oracle.rk_move(kappa, s, n, x0, u)
        sol = solve_ivp(lorentz_rhs(kappa), (0, s), list(x0) + list(u), rtol=1e-12, atol=1e-13 * rho,
                        method="DOP853")
        bound = 1.2e-7 * n * rho + 1e-10 * rho
        assert np.linalg.norm(pos[:2] - sol.y[:2, -1]) < bound
        assert np.linalg.norm(d[:2] - sol.y[3:5, -1]) < 1.2e-7 * n + 1e-10
        assert pos[2] == x0[2] + u[2] * s
        assert d[2] == u[2]
        # the transverse direction keeps its length (rescaled at the end)
        assert math.hypot(d[0], d[1]) == pytest.approx(math.hypot(u[0], u[1]), rel=1e-15)


def test_rk_reduces_to_a_line_along_the_field():
    pos, d = oracle.rk_move(-3.0, 2.5, 7, [1.0, 2.0, 0.0], [0.0, 0.0, 1.0])
    np.testing.assert_array_equal(pos, [1.0, 2.0, 2.5])
    np.testing.assert_array_equal(d, [0.0, 0.0, 1.0])
