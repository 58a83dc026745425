"""Pins for the FP64 oracle: facts fixed by the paper's equations and by
mathematics, checked independently of the oracle's own code.

Each test targets a plausible mistake: a wrong rotation row or sign, a swapped
baseline orientation, a wrong fringe sign, J^dagger C J instead of J C J^dagger
(Eq. 1 vs the form quoted under Eq. 3), a missing horizon cut, a beam with the
wrong width law, a dropped polarisation term.
"""
import math

import numpy as np
import pytest
from scipy import special

from oracle.oracle import (OracleProblem, oracle_enu, oracle_strength, oracle_vis,
                           oracle_voltage, rel_l2)
from paper_2506_02130_gb300 import workloads as W
from tests import _analytic as A

C = 299792458.0
LAT = W.HERA_LATITUDE_RAD


# ---------------------------------------------------------------- rotation
def test_zenith_source():
    s = oracle_enu(1.234, LAT, 1.234, LAT)
    np.testing.assert_allclose(s, [0, 0, 1], atol=1e-15)


def test_celestial_pole_altitude_equals_latitude():
    for lat in (math.radians(40.0), LAT):
        s = oracle_enu(0.7, math.pi / 2, 2.1, lat)
        np.testing.assert_allclose(s, [0, math.cos(lat), math.sin(lat)], atol=1e-15)


def test_equator_source_rises_due_east():
    # hour angle -90 deg: on the horizon, due east, at any latitude
    for lat in (0.3, -0.9):
        lst = 0.4
        s = oracle_enu(lst + math.pi / 2, 0.0, lst, lat)
        np.testing.assert_allclose(s, [1, 0, 0], atol=1e-15)


def test_meridian_transit_north_of_zenith():
    # on the meridian 30 deg north of the zenith: (0, sin 30, cos 30)
    dec = LAT + math.radians(30)
    s = oracle_enu(2.0, dec, 2.0, LAT)
    np.testing.assert_allclose(s, [0, 0.5, math.sqrt(3) / 2], atol=1e-15)


def test_rotation_preserves_angles_and_moves_west():
    rng = np.random.default_rng(0)
    ra, dec = W.uniform_sphere(20, rng)
    eq = np.stack([np.cos(dec) * np.cos(ra), np.cos(dec) * np.sin(ra), np.sin(dec)], 1)
    enu = np.array([oracle_enu(a, d, 0.77, LAT) for a, d in zip(ra, dec)])
    np.testing.assert_allclose(enu @ enu.T, eq @ eq.T, atol=1e-14)
    # a proper rotation (det +1): handedness of the frame is kept
    assert np.linalg.det(enu[:3]) * np.linalg.det(eq[:3]) > 0
    # a transiting source moves west (E decreases) as LST grows
    s0 = oracle_enu(1.0, LAT, 1.0, LAT)
    s1 = oracle_enu(1.0, LAT, 1.001, LAT)
    assert s1[0] < s0[0]


# ---------------------------------------------------------------- beams
def test_gaussian_beam_half_power_at_half_fwhm_scaling_with_frequency():
    fwhm, ref = W.GAUSS_FWHM_150
    for nu in (150e6, 300e6, 100e6):
        theta = 0.5 * fwhm * ref / nu
        assert oracle_voltage("gauss", (fwhm, ref), theta, nu) ** 2 == pytest.approx(0.5, rel=1e-14)
    assert oracle_voltage("gauss", (fwhm, ref), 0.0, 123e6) == 1.0


def test_airy_beam_against_scipy_and_first_null():
    D = 14.0
    rng = np.random.default_rng(1)
    for _ in range(20):
        theta = rng.uniform(1e-3, 1.5)
        nu = rng.uniform(100e6, 200e6)
        x = math.pi * D * nu * math.sin(theta) / C
        assert oracle_voltage("airy", (D,), theta, nu) == pytest.approx(2 * special.j1(x) / x, rel=1e-12, abs=1e-15)
    nu = 150e6
    x0 = special.jn_zeros(1, 1)[0]
    theta0 = math.asin(x0 * C / (math.pi * D * nu))
    assert abs(oracle_voltage("airy", (D,), theta0, nu)) < 1e-12
    assert oracle_voltage("airy", (D,), 0.0, nu) == 1.0


# ---------------------------------------------------------------- coherency (Eq. 1-2)
def _dir_at_az(az, za):
    return np.array([math.sin(za) * math.sin(az), math.sin(za) * math.cos(az), math.cos(za)])


def test_unpolarised_source_gives_identity_coherency():
    s = _dir_at_az(1.1, 0.2)
    A2 = oracle_voltage("airy", (14.0,), 0.2, 150e6) ** 2
    c = oracle_strength("airy", (14.0,), True, s, 150e6, [3.0, 0, 0, 0])
    np.testing.assert_allclose(c, A2 * 3.0 * np.array([1, 0, 0, 1]), atol=1e-14)
    c1 = oracle_strength("airy", (14.0,), False, s, 150e6, [3.0])
    assert c1[0] == pytest.approx(A2 * 3.0, rel=1e-14)


def test_stokes_q_at_45_deg_azimuth_distinguishes_jcjdag_from_jdagcj():
    # R(45) diag(Q,-Q) R(45)^T = [[0, Q], [Q, 0]];  R^T C R would give -Q off-diagonal
    s = _dir_at_az(math.pi / 4, 0.1)
    A2 = oracle_voltage("uniform", (), 0.1, 150e6) ** 2
    c = oracle_strength("uniform", (), True, s, 150e6, [0, 2.0, 0, 0])
    np.testing.assert_allclose(c, A2 * np.array([0, 2.0, 2.0, 0]), atol=1e-14)


def test_stokes_q_due_north_is_diagonal_and_v_is_rotation_invariant():
    s = _dir_at_az(0.0, 0.3)
    c = oracle_strength("uniform", (), True, s, 150e6, [1.0, 0.5, 0, 0])
    np.testing.assert_allclose(c, [1.5, 0, 0, 0.5], atol=1e-15)
    s = _dir_at_az(0.7, 0.3)
    c = oracle_strength("uniform", (), True, s, 150e6, [0, 0, 0, 0.25])
    np.testing.assert_allclose(c, [0, 0.25j, -0.25j, 0], atol=1e-15)


# ---------------------------------------------------------------- direct sum
def _single(ant, pairs, ra, dec, flux, freqs, lst, lat=LAT, beam="uniform", param=(), pol=False):
    return OracleProblem(np.asarray(ant, float), np.asarray(pairs, np.int32), np.atleast_1d(ra),
                         np.atleast_1d(dec), np.asarray(flux, float), np.atleast_1d(freqs),
                         np.atleast_1d(lst), lat, beam, param, pol)


def test_zenith_source_has_zero_phase_on_coplanar_baselines():
    ant = W.hex_array(2)
    pairs = W.cross_pairs(len(ant))
    p = _single(ant, pairs, 0.5, LAT, [[[2.5]]], 150e6, 0.5, beam="gauss", param=W.GAUSS_FWHM_150)
    v = oracle_vis(p)
    np.testing.assert_allclose(v, 2.5, atol=1e-13)


def test_single_source_exact_phase_and_baseline_orientation():
    # source 30 deg north of zenith on the meridian: s = (0, 1/2, sqrt(3)/2).
    # antennas 0 at origin and 1 at 14.6 m north: b_01 = x_0 - x_1 = (0, -14.6, 0)
    ant = [[0, 0, 0], [0, 14.6, 0], [10.0, 0, 0]]
    pairs = [[0, 1], [1, 0], [0, 2]]
    dec = LAT + math.radians(30)
    for nu in (150e6, 187.3e6):
        p = _single(ant, pairs, 2.0, dec, [[[1.0]]], nu, 2.0)
        v = oracle_vis(p, "literal")[0, 0, :, 0]
        phase01 = -2 * math.pi * nu * (-14.6 * 0.5) / C
        np.testing.assert_allclose(v[0], np.exp(1j * phase01), rtol=1e-13)
        np.testing.assert_allclose(v[1], np.exp(-1j * phase01), rtol=1e-13)
        np.testing.assert_allclose(v[2], 1.0, rtol=1e-13)   # east baseline sees no phase


def test_source_below_horizon_contributes_nothing():
    ant = W.hex_array(1)
    pairs = W.cross_pairs(len(ant))
    # celestial north pole from a southern site is below the horizon
    p = _single(ant, pairs, [0.0, 1.0], [math.pi / 2, LAT], [[[5.0], [1.0]]], 150e6, 1.0)
    v = oracle_vis(p)
    np.testing.assert_allclose(v, 1.0, atol=1e-13)


@pytest.fixture(scope="module")
def small():
    return W.config_small(seed=3, n_src=300)


def test_hermitian_and_zero_spacing(small):
    n = len(small.ant_enu)
    pairs = np.array([[i, j] for i in range(n) for j in range(n)], np.int32)
    p = OracleProblem.from_workload(small, pairs=pairs)
    v = oracle_vis(p, "literal")[0, 0, :, 0].reshape(n, n)
    np.testing.assert_array_equal(v, np.conj(v.T))      # odd sine: exact
    from oracle.oracle import oracle_enu as enu
    tot = 0.0
    for k in range(small.sky.n_src):
        s = enu(small.sky.ra[k], small.sky.dec[k], small.lsts_rad[0], LAT)
        if s[2] > 0:
            tot += oracle_voltage("gauss", small.beam_param, math.acos(s[2]), 150e6) ** 2 * small.sky.flux[0, k, 0]
    np.testing.assert_allclose(np.diag(v), tot, rtol=1e-12)


def test_literal_equals_factored_and_translation_invariance(small):
    p = OracleProblem.from_workload(small)
    vl = oracle_vis(p, "literal")
    vf = oracle_vis(p, "factored")
    assert rel_l2(vf, vl) < 1e-13
    p2 = OracleProblem.from_workload(small)
    p2.ant_enu = small.ant_enu + np.array([123.4, -56.7, 0.0])
    assert rel_l2(oracle_vis(p2, "literal"), vl) < 1e-12


def test_baseline_frequency_scaling_invariance_and_linearity():
    rng = np.random.default_rng(5)
    ant = W.hex_array(2, z_sigma_m=0.3, rng=rng)
    pairs = W.cross_pairs(len(ant))
    ra, dec = W.uniform_sphere(200, rng)
    flux = rng.uniform(0.1, 2, (1, 200, 1))
    a = oracle_vis(_single(ant, pairs, ra, dec, flux, 160e6, 0.3), "literal")
    b = oracle_vis(_single(2 * ant, pairs, ra, dec, flux, 80e6, 0.3), "literal")
    assert rel_l2(b, a) < 1e-13
    c = oracle_vis(_single(ant, pairs, ra, dec, 3 * flux, 160e6, 0.3), "literal")
    assert rel_l2(c, 3 * a) < 1e-14


def test_polarised_sum_of_unpolarised_sky_matches_scalar_path():
    rng = np.random.default_rng(6)
    ant = W.hex_array(1)
    pairs = W.cross_pairs(len(ant))
    ra, dec = W.uniform_sphere(100, rng)
    I = rng.uniform(0.1, 2, (100, 2))
    flux4 = np.zeros((4, 100, 2)); flux4[0] = I
    freqs = np.array([120e6, 170e6])
    pol = oracle_vis(_single(ant, pairs, ra, dec, flux4, freqs, 1.0, beam="airy", param=(14.0,), pol=True))
    sc = oracle_vis(_single(ant, pairs, ra, dec, I[None], freqs, 1.0, beam="airy", param=(14.0,)))
    np.testing.assert_allclose(pol[..., 0], sc[..., 0], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(pol[..., 3], sc[..., 0], rtol=1e-13, atol=1e-13)
    assert np.abs(pol[..., 1]).max() < 1e-13 and np.abs(pol[..., 2]).max() < 1e-13


# ---------------------------------------------------------------- analytic diffuse (Section 4.1)
def _diffuse_problem(nside, name, u_wl, nu=150e6):
    # observer at the north pole: zenith angle = 90 deg - dec, no rotation needed
    ra, dec = W.healpix_radec(nside)
    theta = np.pi / 2 - dec
    bright = np.where(theta < np.pi / 2, A.profile(name, np.clip(theta, 0, np.pi / 2)), 0.0)
    flux = (bright * W.healpix_pixel_area(nside))[None, :, None]
    lam = C / nu
    ant = np.zeros((len(u_wl) + 1, 3))
    ant[1:, 0] = -np.asarray(u_wl) * lam * np.cos(0.3)
    ant[1:, 1] = -np.asarray(u_wl) * lam * np.sin(0.3)
    pairs = np.array([[0, k] for k in range(1, len(ant))], np.int32)
    return _single(ant, pairs, ra, dec, flux, nu, 0.9, lat=math.pi / 2)


@pytest.mark.parametrize("name", ["monopole", "quaddome", "gauss"])
def test_analytic_diffuse_converges_with_nside(name):
    u = np.array([0.5, 1.7, 4.2])
    ref = A.monopole(u) if name == "monopole" else A.radial(name, u)
    if name == "monopole":
        np.testing.assert_allclose(A.radial("monopole", u), ref, rtol=1e-10, atol=1e-12)
    errs = []
    for nside in (8, 16, 32):
        v = oracle_vis(_diffuse_problem(nside, name, u))[0, 0, :, 0]
        errs.append(np.abs(v - ref).max())
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < (0.05 if name != "quaddome" else 0.005)
    if name == "quaddome":      # smooth to the horizon: second-order convergence
        assert errs[2] / errs[1] < 0.3
    if name == "monopole":      # horizon cut through a pixel ring: first order
        assert 0.4 < errs[2] / errs[1] < 0.6


def test_golden_fixture_reproduces():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "hex37_oracle.txt")
    rows = np.loadtxt(path)
    prob = W.config_small(seed=11, n_src=40)
    pairs = prob.pairs[::17]
    np.testing.assert_array_equal(rows[:, :2].astype(int), pairs)
    v = oracle_vis(OracleProblem.from_workload(prob, pairs=pairs), "literal")[0, 0, :, 0]
    np.testing.assert_allclose(v, rows[:, 2] + 1j * rows[:, 3], rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------- DFT special case
@pytest.mark.parametrize("N,G,lst", [(16, 5, 0.7), (12, 4, 3.9)])
def test_lattice_sky_reduces_to_numpy_fft2(N, G, lst):
    """Sources on a direction-cosine lattice seen by a grid array: the sum is a
    2-D DFT, evaluated by numpy's FFT (tests/_lattice.py)."""
    from tests._lattice import lattice_case
    L = lattice_case(N=N, G=G, lst=lst)
    enu = np.array([oracle_enu(r, d, lst, L["lat"]) for r, d in zip(L["ra"], L["dec"])])
    np.testing.assert_allclose(enu, L["lmn"], atol=1e-14)
    op = OracleProblem(L["ant"], L["pairs"], L["ra"], L["dec"], L["flux"], L["freqs"], L["lsts"], L["lat"],
                       "uniform", (), False)
    for mode in ("literal", "factored"):
        v = oracle_vis(op, mode)[0, 0, :, 0]
        assert rel_l2(v, L["expected"]) <= 1e-13


# ---------------------------------------------------------------- per-antenna beams (Section 2.2.3)
def _two_beam_problem(polarized=False, seed=11):
    rng = np.random.default_rng(seed)
    ant = W.hex_array(2)
    n = len(ant)
    pairs = W.cross_pairs(n)
    lst = 0.9
    ra, dec = W.visible_hemisphere(60, rng, lst, LAT)
    nst = 4 if polarized else 1
    flux = rng.uniform(0.5, 2.0, (nst, 60, 2))
    if polarized:
        flux[1:] *= 0.2
    beams = [("gauss", (math.radians(30.0), 150e6)), ("gauss", (math.radians(8.0), 150e6)),
             ("airy", (6.0,))] if not polarized else [("airy", (14.0,)), ("airy", (5.0,))]
    boa = rng.integers(0, len(beams), n)
    return OracleProblem(ant, pairs, ra, dec, flux, np.array([120e6, 180e6]), np.array([lst]), LAT,
                         "gauss", (math.radians(10.0), 150e6), polarized, beams, boa)


def test_per_antenna_beams_one_beam_equals_the_shared_beam():
    p = _two_beam_problem()
    p.beams = [("gauss", (math.radians(10.0), 150e6))]
    p.beam_of_ant = np.zeros(len(p.ant_enu), dtype=int)
    v1 = oracle_vis(p)
    p.beam_of_ant = None
    v0 = oracle_vis(p)
    assert rel_l2(v1, v0) <= 1e-14


def test_per_antenna_beams_single_source_is_the_product_of_the_two_voltages():
    """One source: V_ij = A_b(i)(theta) A_b(j)(theta) I exp(-2 pi i nu b.s / c), with the voltage of
    each antenna's own beam (a swapped or shared assignment fails)."""
    p = _two_beam_problem()
    p.ra, p.dec, p.flux = p.ra[:1], p.dec[:1], p.flux[:, :1]
    v = oracle_vis(p, "literal")
    s = oracle_enu(p.ra[0], p.dec[0], p.lsts_rad[0], LAT)
    theta = math.acos(s[2])
    for f, nu in enumerate(p.freqs_hz):
        A = [oracle_voltage(k, par, theta, nu) for k, par in p.beams]
        for b, (i, j) in enumerate(p.pairs):
            bvec = p.ant_enu[i] - p.ant_enu[j]
            want = (A[p.beam_of_ant[i]] * A[p.beam_of_ant[j]] * p.flux[0, 0, f]
                    * np.exp(-2j * math.pi * nu * np.dot(bvec, s) / C))
            assert abs(v[f, 0, b, 0] - want) <= 1e-13 * abs(p.flux[0, 0, f])


def test_per_antenna_beams_hermitian_and_factored_equals_literal():
    p = _two_beam_problem()
    lit = oracle_vis(p, "literal")
    fac = oracle_vis(p, "factored")
    assert rel_l2(fac, lit) <= 1e-13
    q = OracleProblem(**{**p.__dict__, "pairs": p.pairs[:, ::-1].copy()})
    assert np.array_equal(oracle_vis(q, "literal"), np.conj(lit))


def test_per_antenna_beams_polarised_is_Ji_C_Jj_dagger():
    """Polarised single source with different Airy dishes: the four products are J_i C J_j^dagger,
    checked against numpy 2x2 matrix products (J = A R(az))."""
    p = _two_beam_problem(polarized=True)
    p.ra, p.dec, p.flux = p.ra[:1], p.dec[:1], p.flux[:, :1]
    v = oracle_vis(p, "literal")
    s = oracle_enu(p.ra[0], p.dec[0], p.lsts_rad[0], LAT)
    theta, az = math.acos(s[2]), math.atan2(s[0], s[1])
    R = np.array([[math.cos(az), -math.sin(az)], [math.sin(az), math.cos(az)]])
    for f, nu in enumerate(p.freqs_hz):
        I, Q, U, V = p.flux[:, 0, f]
        Cm = np.array([[I + Q, U + 1j * V], [U - 1j * V, I - Q]])
        A = [oracle_voltage(k, par, theta, nu) for k, par in p.beams]
        for b, (i, j) in enumerate(p.pairs):
            Ji, Jj = A[p.beam_of_ant[i]] * R, A[p.beam_of_ant[j]] * R
            M = Ji @ Cm @ Jj.conj().T
            ph = np.exp(-2j * math.pi * nu * np.dot(p.ant_enu[i] - p.ant_enu[j], s) / C)
            np.testing.assert_allclose(v[f, 0, b], M.ravel() * ph, rtol=0, atol=1e-12 * I)


# ---------------------------------------------------------------- gridded beams (Section 2.4)
def test_grid_beam_nodes_rows_and_azimuth_wrap():
    from oracle.oracle import oracle_voltage_grid
    rng = np.random.default_rng(21)
    nth, nph = 7, 6
    T = rng.uniform(0.1, 1.0, size=(nth, nph))
    dth, dph = (math.pi / 2) / (nth - 1), 2 * math.pi / nph
    for i in range(nth - 1):
        for j in range(nph):
            assert oracle_voltage_grid(T, i * dth, j * dph) == pytest.approx(T[i, j], abs=1e-15)
    # halfway between two rows, on a column: the mean of the two samples
    assert oracle_voltage_grid(T, 2.5 * dth, 4 * dph) == pytest.approx(0.5 * (T[2, 4] + T[3, 4]), abs=1e-14)
    # the azimuth is periodic: between the last column and column 0, from either side of 2 pi
    mid = 0.5 * (T[3, nph - 1] + T[3, 0])
    assert oracle_voltage_grid(T, 3 * dth, 2 * math.pi - 0.5 * dph) == pytest.approx(mid, abs=1e-14)
    assert oracle_voltage_grid(T, 3 * dth, -0.5 * dph) == pytest.approx(mid, abs=1e-14)
    # linear in theta and constant in azimuth is reproduced exactly anywhere
    L = np.repeat((0.9 - 0.4 * np.arange(nth) * dth)[:, None], nph, axis=1)
    for th, az in [(0.123, 0.3), (1.4, 5.9), (0.77, 2.2)]:
        assert oracle_voltage_grid(L, th, az) == pytest.approx(0.9 - 0.4 * th, abs=1e-14)


def test_grid_beam_azimuth_is_measured_east_of_north():
    from oracle.oracle import oracle_voltage_grid
    freqs = np.array([150e6])
    G = W.grid_beam(freqs, 361, 360, math.radians(20.0), 150e6, ellipticity=0.4)[0]
    th = math.radians(12.0)
    # due north (az 0) the pattern is 1.4x wider than due east (az 90 deg): compare the two directions
    for az, e in [(0.0, 1.4), (math.pi / 2, 0.6)]:
        fwhm = math.radians(20.0) * e
        want = math.sqrt(math.exp(-4 * math.log(2) * th ** 2 / fwhm ** 2))
        assert oracle_voltage_grid(G, th, az) == pytest.approx(want, rel=2e-4)
    # the ENU direction of a source east of the zenith has az = 90 deg: E = sin(th), N = 0
    s_east = np.array([math.sin(th), 0.0, math.cos(th)])
    assert math.atan2(s_east[0], s_east[1]) == pytest.approx(math.pi / 2)


def test_grid_beam_visibilities_converge_to_the_analytic_beam_at_second_order():
    prob = W.config_hex127(seed=22, n_chan=2, n_time=1, n_point=400, nside=0, radius=2)
    prob.beam_param = (math.radians(30.0), 150e6)
    ref = oracle_vis(OracleProblem.from_workload(prob), "literal")
    errs = []
    for nth in (46, 91, 181):
        p = OracleProblem.from_workload(prob)
        p.beam = "grid"
        p.beam_grids = {-1: W.grid_beam(prob.freqs_hz, nth, 4, math.radians(30.0), 150e6)}
        errs.append(rel_l2(oracle_vis(p, "literal"), ref))
    assert errs[0] < 1e-2
    for a, b in zip(errs, errs[1:]):
        assert 3.0 < a / b < 5.0, errs


def test_grid_beam_as_one_of_two_per_antenna_beams():
    prob = W.config_hex127(seed=23, n_chan=2, n_time=1, n_point=300, nside=0, radius=2)
    boa = np.arange(len(prob.ant_enu)) % 2
    analytic = OracleProblem.from_workload(prob)
    analytic.beams = [("gauss", (math.radians(25.0), 150e6)), ("airy", (6.0,))]
    analytic.beam_of_ant = boa
    gridded = OracleProblem.from_workload(prob)
    gridded.beams = [("grid", ()), ("airy", (6.0,))]
    gridded.beam_of_ant = boa
    gridded.beam_grids = {0: W.grid_beam(prob.freqs_hz, 721, 4, math.radians(25.0), 150e6)}
    assert rel_l2(oracle_vis(gridded, "literal"), oracle_vis(analytic, "literal")) < 2e-5
    assert rel_l2(oracle_vis(gridded, "factored"), oracle_vis(gridded, "literal")) < 1e-12


def test_bicubic_grid_beam_interpolates_and_matches_scipy_splines_per_axis():
    from scipy import ndimage
    from oracle.oracle import oracle_voltage_grid3
    rng = np.random.default_rng(24)
    nth, nph = 9, 10
    dth, dph = (math.pi / 2) / (nth - 1), 2 * math.pi / nph
    T = rng.uniform(0.2, 1.0, size=(nth, nph))
    for i in range(nth - 1):
        for j in range(nph):
            assert oracle_voltage_grid3(T, i * dth, j * dph) == pytest.approx(T[i, j], abs=1e-12)
    # zenith-angle axis: the cubic spline with whole-sample mirror ends (scipy's 'mirror')
    f = rng.uniform(0.2, 1.0, nth)
    A = np.repeat(f[:, None], nph, axis=1)
    for u in (0.2, 0.5, 3.7, 6.01, 7.9):
        want = ndimage.map_coordinates(f, [[u]], order=3, mode="mirror")[0]
        assert oracle_voltage_grid3(A, u * dth, 1.234) == pytest.approx(want, abs=1e-12)
    # azimuth axis: the periodic cubic spline (scipy's 'grid-wrap'), on both sides of 2 pi
    g = rng.uniform(0.2, 1.0, nph)
    P = np.repeat(g[None, :], nth, axis=0)
    for v in (0.3, 4.5, 9.2, 9.9):
        want = ndimage.map_coordinates(g, [[v]], order=3, mode="grid-wrap")[0]
        assert oracle_voltage_grid3(P, 0.4, v * dph) == pytest.approx(want, abs=1e-12)
        assert oracle_voltage_grid3(P, 0.4, v * dph - 2 * math.pi) == pytest.approx(want, abs=1e-12)
    # a separable table gives the product of the two one-axis splines
    S = np.outer(f, g)
    for u, v in ((1.3, 2.6), (7.5, 9.7)):
        want = (ndimage.map_coordinates(f, [[u]], order=3, mode="mirror")[0] *
                ndimage.map_coordinates(g, [[v]], order=3, mode="grid-wrap")[0])
        assert oracle_voltage_grid3(S, u * dth, v * dph) == pytest.approx(want, abs=1e-12)


def test_bicubic_grid_beam_converges_at_fourth_order():
    prob = W.config_hex127(seed=25, n_chan=2, n_time=1, n_point=400, nside=0, radius=2)
    prob.beam_param = (math.radians(30.0), 150e6)
    ref = oracle_vis(OracleProblem.from_workload(prob), "literal")
    errs = []
    for nth in (46, 91, 181):
        p = OracleProblem.from_workload(prob)
        p.beam, p.beam_grid_order = "grid", 3
        p.beam_grids = {-1: W.grid_beam(prob.freqs_hz, nth, 4, math.radians(30.0), 150e6)}
        errs.append(rel_l2(oracle_vis(p, "literal"), ref))
    # fourth order: a factor 16 per halving of the grid step (second order, bilinear, gives 4)
    assert 11.0 < math.sqrt(errs[0] / errs[2]) < 23.0, errs
