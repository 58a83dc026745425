"""Per-antenna beams (Section 2.2.3): one transform per unordered pair of
beams, on both routes, against the oracle's J_i C J_j^dagger."""
import math

import numpy as np
import pytest

from oracle.oracle import OracleProblem, oracle_vis, rel_l2
from paper_2506_02130_gb300 import fv, workloads as W

pytestmark = pytest.mark.gpu

TOL = {fv.FV_FP64: 1e-9, fv.FV_MIXED: 2e-5}
EPS = {fv.FV_FP64: 1e-11, fv.FV_MIXED: 1e-6}
THREE = [("gauss", (math.radians(12.0), 150e6)), ("gauss", (math.radians(7.0), 150e6)), ("airy", (9.0,))]


def _run(prob, precision, transform, beams=None, boa=None, beams_after_sky=False):
    p = fv.Plan.create(prob.freqs_hz, prob.lsts_rad, prob.latitude_rad, prob.beam, prob.beam_param, precision,
                       EPS[precision], prob.polarized, transform=transform)
    p.set_array(prob.ant_enu, prob.pairs)
    if beams is not None and not beams_after_sky:
        p.set_beams(beams, boa)
    p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
    if beams is not None and beams_after_sky:
        p.set_beams(beams, boa)
    out = p.run()
    info = p.info()
    p.close()
    return out, info


def _with_beams(prob, beams, seed=0):
    prob.beams = beams
    prob.beam_of_ant = np.random.default_rng(seed).integers(0, len(beams), len(prob.ant_enu))
    return prob


@pytest.mark.parametrize("transform", ["type3", "lattice"])
@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
def test_three_beams_match_oracle(precision, transform):
    prob = W.config_hex127(seed=71, n_chan=3, n_time=2, n_point=600, nside=4, radius=3)
    if transform == "lattice":
        prob.ant_enu = W.hex_array(3)
    _with_beams(prob, THREE, seed=1)
    out, info = _run(prob, precision, transform, prob.beams, prob.beam_of_ant)
    assert info["transform"] == transform
    present = {tuple(sorted((prob.beam_of_ant[i], prob.beam_of_ant[j]))) for i, j in prob.pairs}
    assert info["beam_groups"] == len(present) == 6
    assert rel_l2(out, oracle_vis(OracleProblem.from_workload(prob))) <= TOL[precision]


@pytest.mark.parametrize("transform", ["type3", "lattice"])
def test_polarised_airy_dishes_of_two_sizes(transform):
    prob = W.config_hex350_pol(seed=72, n_chan=2, n_time=1, n_point=300, nside=4, n_keep=None, radius=2)
    _with_beams(prob, [("airy", (14.0,)), ("airy", (6.0,))], seed=2)
    out, info = _run(prob, fv.FV_MIXED, transform, prob.beams, prob.beam_of_ant, beams_after_sky=True)
    assert info["beam_groups"] == 3
    ref = oracle_vis(OracleProblem.from_workload(prob))
    for p in range(4):
        assert rel_l2(out[..., p], ref[..., p]) <= 4e-5, p


def test_one_beam_for_all_equals_the_shared_beam_and_reset():
    prob = W.config_small(seed=73, n_src=300)
    base, info0 = _run(prob, fv.FV_FP64, "type3")
    same, info1 = _run(prob, fv.FV_FP64, "type3", [("gauss", prob.beam_param)], np.zeros(len(prob.ant_enu), int))
    assert info0["beam_groups"] == info1["beam_groups"] == 1
    assert rel_l2(same, base) <= 1e-13
    # clearing the beams returns to the plan's beam
    p = fv.Plan.from_problem(prob, precision=fv.FV_FP64, eps=1e-11, transform="type3")
    p.set_beams(THREE, np.arange(len(prob.ant_enu)) % 3)
    assert p.info()["beam_groups"] == 6
    p.set_beams(None, None)
    p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
    assert p.info()["beam_groups"] == 1
    assert rel_l2(p.run(), base) <= 1e-13
    p.close()


def test_set_beams_errors():
    prob = W.config_small(seed=74, n_src=50)
    p = fv.Plan.create(prob.freqs_hz, prob.lsts_rad, prob.latitude_rad, prob.beam, prob.beam_param, fv.FV_FP64, 1e-10)
    with pytest.raises(fv.FvError) as ei:
        p.set_beams(THREE, np.zeros(37, int))
    assert ei.value.status == fv.FV_ERR_STATE
    p.set_array(prob.ant_enu, prob.pairs)
    with pytest.raises(fv.FvError) as ei:
        p.set_beams(THREE, np.full(37, 3))
    assert ei.value.status == fv.FV_ERR_ARG
    with pytest.raises(fv.FvError) as ei:
        p.set_beams([("airy", (-1.0,))], np.zeros(37, int))
    assert ei.value.status == fv.FV_ERR_ARG
    p.close()
