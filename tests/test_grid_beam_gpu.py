"""Gridded (numerical) beams of Section 2.4 on the GPU: voltage samples per
channel on a zenith-angle x azimuth grid, interpolated bilinearly, on every
route, against the oracle's own bilinear interpolation of the same samples."""
import math

import numpy as np
import pytest

from oracle.basis import basis_vis
from oracle.oracle import OracleProblem, oracle_vis, rel_l2
from paper_2506_02130_gb300 import fv, workloads as W

pytestmark = pytest.mark.gpu

TOL = {fv.FV_FP64: 1e-9, fv.FV_MIXED: 2e-5}
EPS = {fv.FV_FP64: 1e-11, fv.FV_MIXED: 1e-6}


def _gridded(prob, n_theta=46, n_phi=24, fwhm_deg=25.0, ellipticity=0.35, order=1):
    prob.beam = "grid"
    prob.beam_param = ()
    prob.beam_grid_order = order
    prob.beam_grids = {-1: W.grid_beam(prob.freqs_hz, n_theta, n_phi, math.radians(fwhm_deg), 150e6,
                                       ellipticity=ellipticity)}
    return prob


def _run(prob, precision, transform, **kw):
    p = fv.Plan.from_problem(prob, precision=precision, eps=EPS[precision], transform=transform, **kw)
    if prob.beams is not None:
        p.set_beams(prob.beams, prob.beam_of_ant, prob.beam_grids, prob.beam_grid_order)
    p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
    out = p.run()
    info = p.info()
    p.close()
    return out, info


@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
def test_type3_gridded_beam_matches_oracle(precision):
    prob = _gridded(W.config_hex127(seed=91, n_chan=3, n_time=2, n_point=700, nside=4, radius=3))
    out, info = _run(prob, precision, "type3")
    assert info["transform"] == "type3"
    assert rel_l2(out, oracle_vis(OracleProblem.from_workload(prob))) <= TOL[precision]


def test_lattice_route_gridded_beam():
    prob = _gridded(W.config_hex127(seed=92, n_chan=3, n_time=2, n_point=600, nside=4, radius=3))
    prob.ant_enu = W.hex_array(3)
    out, info = _run(prob, fv.FV_MIXED, "lattice")
    assert info["transform"] == "lattice"
    assert rel_l2(out, oracle_vis(OracleProblem.from_workload(prob))) <= TOL[fv.FV_MIXED]


def test_basis_route_gridded_beam():
    prob = _gridded(W.config_hex127(seed=93, n_chan=8, n_time=1, n_point=500, nside=2, radius=2),
                    fwhm_deg=40.0)
    out, _ = _run(prob, fv.FV_MIXED, "basis", n_basis=5)
    assert rel_l2(out, basis_vis(OracleProblem.from_workload(prob), 5)) <= TOL[fv.FV_MIXED]


def test_polarised_gridded_and_analytic_per_antenna_beams():
    prob = W.config_hex350_pol(seed=94, n_chan=2, n_time=1, n_point=300, nside=4, n_keep=None, radius=2)
    prob.beams = [("grid", ()), ("airy", (6.0,))]
    prob.beam_of_ant = np.arange(len(prob.ant_enu)) % 2
    prob.beam_grids = {0: W.grid_beam(prob.freqs_hz, 61, 36, math.radians(20.0), 150e6, ellipticity=0.2)}
    out, info = _run(prob, fv.FV_MIXED, "type3")
    assert info["beam_groups"] == 3
    ref = oracle_vis(OracleProblem.from_workload(prob))
    for p in range(4):
        assert rel_l2(out[..., p], ref[..., p]) <= 4e-5, p


def test_fine_grid_of_the_analytic_beam_reproduces_the_analytic_plan():
    prob = W.config_hex127(seed=95, n_chan=2, n_time=1, n_point=500, nside=0, radius=2)
    prob.beam_param = (math.radians(25.0), 150e6)
    analytic, _ = _run(prob, fv.FV_FP64, "type3")
    gridded, _ = _run(_gridded(prob, n_theta=1801, n_phi=4, ellipticity=0.0), fv.FV_FP64, "type3")
    assert rel_l2(gridded, analytic) < 1e-5


def test_beam_grid_set_after_the_sky_and_errors():
    prob = W.config_small(seed=96, n_src=300)
    grid = W.grid_beam(prob.freqs_hz, 31, 12, math.radians(15.0), 150e6, ellipticity=0.3)
    p = fv.Plan.from_problem(prob, precision=fv.FV_MIXED, eps=1e-6, transform="type3")
    p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
    p.run()
    p.set_beam_grid(-1, grid)
    out = p.run()
    prob.beam, prob.beam_param, prob.beam_grids = "grid", (), {-1: grid}
    assert rel_l2(out, oracle_vis(OracleProblem.from_workload(prob))) <= TOL[fv.FV_MIXED]
    lib = fv.load_library()
    g = np.ascontiguousarray(grid)
    assert lib.fv_set_beam_grid(p.handle, 0, 31, 12, 1, g.ctypes.data) == fv.FV_ERR_ARG    # no per-antenna beams
    assert lib.fv_set_beam_grid(p.handle, -1, 1, 12, 1, g.ctypes.data) == fv.FV_ERR_ARG    # n_theta < 2
    assert lib.fv_set_beam_grid(p.handle, -1, 31, 12, 2, g.ctypes.data) == fv.FV_ERR_ARG   # order 2
    bad = g.copy()
    bad[0, 3, 4] = np.nan
    assert lib.fv_set_beam_grid(p.handle, -1, 31, 12, 1, bad.ctypes.data) == fv.FV_ERR_ARG
    p.close()
    with pytest.raises(fv.FvError) as e:
        fv.Plan.create(prob.freqs_hz, prob.lsts_rad, prob.latitude_rad, beam="grid")
    assert e.value.status == fv.FV_ERR_ARG


def test_axisymmetric_grid_one_azimuth_column_fp64():
    prob = _gridded(W.config_hex127(seed=97, n_chan=2, n_time=1, n_point=500, nside=2, radius=2),
                    n_theta=91, n_phi=1, ellipticity=0.0)
    out, _ = _run(prob, fv.FV_FP64, "type3")
    assert rel_l2(out, oracle_vis(OracleProblem.from_workload(prob))) <= TOL[fv.FV_FP64]


@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
def test_bicubic_gridded_beam_type3(precision):
    prob = _gridded(W.config_hex127(seed=98, n_chan=3, n_time=2, n_point=700, nside=4, radius=3), order=3)
    out, _ = _run(prob, precision, "type3")
    assert rel_l2(out, oracle_vis(OracleProblem.from_workload(prob))) <= TOL[precision]


def test_bicubic_per_antenna_gridded_beam_on_the_basis_and_lattice_routes():
    prob = W.config_hex127(seed=99, n_chan=6, n_time=1, n_point=500, nside=2, radius=3)
    prob.ant_enu = W.hex_array(3)
    prob.beams = [("grid", ()), ("gauss", (math.radians(30.0), 150e6))]
    prob.beam_of_ant = np.arange(len(prob.ant_enu)) % 2
    prob.beam_grids = {0: W.grid_beam(prob.freqs_hz, 31, 16, math.radians(35.0), 150e6, ellipticity=0.25)}
    prob.beam_grid_order = 3
    ref = oracle_vis(OracleProblem.from_workload(prob))
    out, _ = _run(prob, fv.FV_MIXED, "lattice")
    assert rel_l2(out, ref) <= TOL[fv.FV_MIXED]
    out, _ = _run(prob, fv.FV_MIXED, "basis", n_basis=4)
    assert rel_l2(out, basis_vis(OracleProblem.from_workload(prob), 4)) <= TOL[fv.FV_MIXED]


def test_bicubic_fine_grid_is_closer_to_the_analytic_beam_than_bilinear():
    prob = W.config_hex127(seed=100, n_chan=2, n_time=1, n_point=500, nside=0, radius=2)
    prob.beam_param = (math.radians(25.0), 150e6)
    analytic, _ = _run(prob, fv.FV_FP64, "type3")
    lin, _ = _run(_gridded(prob, n_theta=181, n_phi=4, ellipticity=0.0, order=1), fv.FV_FP64, "type3")
    cub, _ = _run(_gridded(prob, n_theta=181, n_phi=4, ellipticity=0.0, order=3), fv.FV_FP64, "type3")
    assert rel_l2(cub, analytic) < 0.05 * rel_l2(lin, analytic)
