"""Spectral-basis route (Appendix A) on the GPU against the basis oracle:
the same basis truncation evaluated by FP64 direct sums, so the two agree to
the NUFFT tolerance; with a complete basis both equal the plain direct sum."""
import math

import numpy as np
import pytest
import torch

from oracle.basis import basis_vis
from oracle.oracle import OracleProblem, oracle_vis, rel_l2
from paper_2506_02130_gb300 import fv, workloads as W

pytestmark = pytest.mark.gpu

TOL = {fv.FV_FP64: 1e-9, fv.FV_MIXED: 2e-5}
EPS = {fv.FV_FP64: 1e-11, fv.FV_MIXED: 1e-6}


def _problem(seed=81, n_chan=8, n_time=2, n_point=500, nside=4, radius=2, fwhm_deg=40.0, coplanar=False):
    prob = W.config_hex127(seed=seed, n_chan=n_chan, n_time=n_time, n_point=n_point, nside=nside, radius=radius)
    prob.beam_param = (math.radians(fwhm_deg), 150e6)
    if coplanar:
        prob.ant_enu = prob.ant_enu.copy()
        prob.ant_enu[:, 2] = 0.0
    return prob


def _run(prob, precision, K, beams=None, boa=None, **kw):
    p = fv.Plan.create(prob.freqs_hz, prob.lsts_rad, prob.latitude_rad, prob.beam, prob.beam_param, precision,
                       EPS[precision], prob.polarized, transform="basis", n_basis=K, **kw)
    p.set_array(prob.ant_enu, prob.pairs)
    if beams is not None:
        p.set_beams(beams, boa)
    p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
    out = p.run()
    info = p.info()
    p.close()
    return out, info


@pytest.mark.parametrize("coplanar", [False, True])
@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
def test_basis_route_matches_the_basis_oracle(precision, coplanar):
    prob = _problem(coplanar=coplanar)
    K = 4
    out, info = _run(prob, precision, K)
    assert info["transform"] == "basis" and info["basis_terms"] == K
    assert info["dims"] == (2 if coplanar else 3)
    ref = basis_vis(OracleProblem.from_workload(prob), K)
    assert rel_l2(out, ref) <= TOL[precision]
    # per channel too: no channel is sacrificed to the others
    for q in range(len(prob.freqs_hz)):
        assert rel_l2(out[q], ref[q]) <= 3 * TOL[precision], q


@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
def test_complete_basis_is_the_direct_sum(precision):
    prob = _problem(seed=82, n_chan=6, n_time=1)
    out, _ = _run(prob, precision, 6)
    assert rel_l2(out, oracle_vis(OracleProblem.from_workload(prob), "literal")) <= TOL[precision]


def test_ragged_sizes_and_odd_K():
    # 5 basis functions (three padded spreading planes), 13 channels, 37 antennas
    prob = _problem(seed=83, n_chan=13, n_time=3, n_point=333, nside=2, radius=3)
    out, info = _run(prob, fv.FV_MIXED, 5)
    assert info["basis_grid"][0] > 0
    assert rel_l2(out, basis_vis(OracleProblem.from_workload(prob), 5)) <= TOL[fv.FV_MIXED]


def test_per_antenna_beams_one_transform_per_pair():
    prob = _problem(seed=84, n_chan=5, n_time=1, n_point=400)
    prob.beams = [("gauss", (math.radians(35.0), 150e6)), ("airy", (5.0,))]
    prob.beam_of_ant = np.arange(len(prob.ant_enu)) % 2
    out, info = _run(prob, fv.FV_MIXED, 3, prob.beams, prob.beam_of_ant)
    assert info["beam_groups"] == 3
    assert rel_l2(out, basis_vis(OracleProblem.from_workload(prob), 3)) <= TOL[fv.FV_MIXED]


def test_flux_rewritten_in_place_between_executions():
    prob = _problem(seed=85, n_chan=6, n_time=1, n_point=300, nside=0)
    p = fv.Plan.create(prob.freqs_hz, prob.lsts_rad, prob.latitude_rad, prob.beam, prob.beam_param, fv.FV_MIXED,
                       1e-6, False, transform="basis", n_basis=3)
    p.set_array(prob.ant_enu, prob.pairs)
    flux = torch.tensor(prob.sky.flux, dtype=torch.float32, device="cuda")
    p.set_sky(prob.sky.ra, prob.sky.dec, flux)
    a = p.run().copy()
    flux.mul_(2.0)
    b = p.run()
    p.close()
    assert rel_l2(b, 2.0 * a) <= 1e-6
    assert rel_l2(a, basis_vis(OracleProblem.from_workload(prob), 3)) <= TOL[fv.FV_MIXED]


def test_errors():
    prob = _problem(seed=86, n_chan=4, n_time=1, n_point=50, nside=0)
    for K in (5, -1):
        with pytest.raises(fv.FvError) as e:
            fv.Plan.create(prob.freqs_hz, prob.lsts_rad, prob.latitude_rad, transform="basis", n_basis=K)
        assert e.value.status == fv.FV_ERR_ARG
    with pytest.raises(fv.FvError) as e:
        fv.Plan.create(prob.freqs_hz, prob.lsts_rad, prob.latitude_rad, polarized=True, transform="basis",
                       n_basis=2)
    assert e.value.status == fv.FV_ERR_UNSUPPORTED
    # repeated channel frequencies cannot carry more basis functions than distinct frequencies
    p = fv.Plan.create(np.array([150e6, 150e6, 160e6]), prob.lsts_rad, prob.latitude_rad, transform="basis",
                       n_basis=3)
    p.set_array(prob.ant_enu, prob.pairs)
    with pytest.raises(fv.FvError) as e:
        p.set_sky(prob.sky.ra, prob.sky.dec, np.ascontiguousarray(prob.sky.flux[:, :, :3]))
    assert e.value.status == fv.FV_ERR_ARG
    p.close()
    # whole times only: batches and the static entry refuse a basis plan
    p = fv.Plan.create(prob.freqs_hz, prob.lsts_rad, prob.latitude_rad, prob.beam, prob.beam_param, fv.FV_MIXED,
                       1e-6, transform="basis", n_basis=2)
    p.set_array(prob.ant_enu, prob.pairs)
    p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
    out = torch.empty(p.out_shape, dtype=torch.complex64, device="cuda")
    b = fv.Batch(device=0)
    with pytest.raises(fv.FvError) as e:
        b.add(p, out)
    assert e.value.status == fv.FV_ERR_UNSUPPORTED
    b.close()
    with pytest.raises(fv.FvError) as e:
        fv.fv_execute_static(p.handle, out)
    assert e.value.status == fv.FV_ERR_UNSUPPORTED
    p.close()


def test_empty_and_invisible_skies_and_a_single_time():
    prob = _problem(seed=87, n_chan=4, n_time=1, n_point=50, nside=0)
    n_f = len(prob.freqs_hz)
    prob.sky = W.Sky(np.zeros(0), np.zeros(0), np.zeros((1, 0, n_f)))
    out, _ = _run(prob, fv.FV_MIXED, 2)
    assert np.all(out == 0)
    prob.sky = W.Sky(np.array([0.1, 2.0]), np.array([np.pi / 2, np.pi / 2 - 1e-3]), np.ones((1, 2, n_f)))
    out, _ = _run(prob, fv.FV_FP64, 3)      # around the north celestial pole: below the horizon at -30.7 deg
    assert np.all(out == 0)


@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
def test_single_channel_single_basis_function_is_the_direct_sum(precision):
    prob = _problem(seed=88, n_chan=1, n_time=2, n_point=400, nside=2)
    out, info = _run(prob, precision, 1)
    assert info["basis_terms"] == 1
    assert rel_l2(out, oracle_vis(OracleProblem.from_workload(prob), "literal")) <= TOL[precision]


def test_automatic_K_is_the_degree_of_a_polynomial_sky():
    prob = _problem(seed=89, n_chan=9, n_time=2, n_point=300, nside=0)
    prob.beam, prob.beam_param = "uniform", ()
    x = (prob.freqs_hz - 150e6) / 50e6
    a = np.random.default_rng(3).uniform(0.5, 2.0, size=(prob.sky.n_src, 3))
    prob.sky.flux = (a[:, :1] + a[:, 1:2] * x[None] - 0.3 * a[:, 2:3] * x[None] ** 2)[None]
    out, info = _run(prob, fv.FV_MIXED, 0)
    assert info["basis_terms"] == 3
    assert info["basis_fit_error"] < 1e-7          # the squared-norm estimate resolves about 1e-8
    assert rel_l2(out, oracle_vis(OracleProblem.from_workload(prob), "literal")) <= TOL[fv.FV_MIXED]


def test_automatic_K_meets_eps_on_a_power_law_sky_through_the_beam():
    prob = _problem(seed=90, n_chan=16, n_time=2, n_point=800, nside=4, fwhm_deg=20.0)
    out, info = _run(prob, fv.FV_MIXED, 0)
    assert 1 < info["basis_terms"] <= 16
    assert 0.0 <= info["basis_fit_error"] <= EPS[fv.FV_MIXED]
    assert rel_l2(out, oracle_vis(OracleProblem.from_workload(prob), "literal")) <= TOL[fv.FV_MIXED]
    # an explicit K reports no fit
    _, info = _run(prob, fv.FV_MIXED, 4)
    assert info["basis_fit_error"] == -1.0


def test_sixteen_basis_functions_over_32_channels():
    # the largest basis: K * Nz = 128 values per cell, four loads per footprint tap
    prob = _problem(seed=91, n_chan=32, n_time=1, n_point=400, nside=2)
    out, info = _run(prob, fv.FV_MIXED, 16)
    assert info["basis_terms"] == 16
    assert rel_l2(out, basis_vis(OracleProblem.from_workload(prob), 16)) <= TOL[fv.FV_MIXED]
