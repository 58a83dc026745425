"""Height terms of a non-coplanar array on the type-3 route (Section 2.2.2: the up
axis of a nearly flat array), against the FP64 oracle through the C ABI.

The height factor exp(-i k b_up n) of a slice is expanded in Chebyshev terms of
the sources' up component, so a slice becomes K two-dimensional transforms whose
targets sum them with Bessel weights.  The array here is a hexagon with
horizontal and vertical jitter, so it is neither coplanar nor a lattice.
Tolerances as for every other route: 2e-5 (mixed) and 1e-9 (FP64) relative L2.
"""
import numpy as np
import pytest

from oracle.oracle import OracleProblem, oracle_vis, rel_l2
from paper_2506_02130_gb300 import fv, workloads as W

pytestmark = pytest.mark.gpu

TOL = {fv.FV_FP64: 1e-9, fv.FV_MIXED: 2e-5}
EPS = {fv.FV_FP64: 1e-11, fv.FV_MIXED: 1e-6}


def _jittered(seed, radius=4, xy_sigma=0.4, z_sigma=0.05, n_chan=4, n_time=2, n_point=1500, nside=8,
              polarised=False):
    """A hexagon whose antennas are moved by Gaussian offsets: xy_sigma (m) horizontally, z_sigma (m) up."""
    if polarised:
        prob = W.config_hex350_pol(seed=seed, n_chan=n_chan, n_time=n_time, n_point=n_point, nside=nside,
                                   n_keep=None, radius=radius)
    else:
        prob = W.config_hex127(seed=seed, n_chan=n_chan, n_time=n_time, n_point=n_point, nside=nside,
                               radius=radius)
    rng = np.random.default_rng(seed + 1000)
    ant = W.hex_array(radius)
    ant[:, :2] += rng.normal(0.0, xy_sigma, (len(ant), 2))
    ant[:, 2] = rng.normal(0.0, z_sigma, len(ant))
    prob.ant_enu = ant
    return prob


def _run(prob, precision, heights, eps=None, **kw):
    p = fv.Plan.create(prob.freqs_hz, prob.lsts_rad, prob.latitude_rad, prob.beam, prob.beam_param, precision,
                       EPS[precision] if eps is None else eps, prob.polarized, transform="type3",
                       heights=heights, **kw)
    try:
        p.set_array(prob.ant_enu, prob.pairs)
        p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
        out = p.run()
        info = p.info()
    finally:
        p.close()
    return out, info


@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
def test_height_terms_match_oracle_on_a_jittered_non_lattice_array(precision):
    prob = _jittered(71)
    assert fv.fv_lattice_detect(prob.ant_enu) is None         # not a lattice (and not coplanar)
    out, info = _run(prob, precision, "terms")
    assert info["dims"] == 2 and info["height_terms"] >= 2 and not info["lattice"]
    ref = oracle_vis(OracleProblem.from_workload(prob))
    err = rel_l2(out, ref)
    assert err <= TOL[precision], err
    for f in range(out.shape[0]):                              # no slice is sacrificed to the others
        for t in range(out.shape[1]):
            assert rel_l2(out[f, t], ref[f, t]) <= 3 * TOL[precision], (f, t)
    # the three-dimensional grid on the same problem: same answer
    out3, info3 = _run(prob, precision, "grid")
    assert info3["dims"] == 3 and info3["height_terms"] == 0
    assert rel_l2(out3, ref) <= TOL[precision]
    assert rel_l2(out, out3) <= 2 * TOL[precision]


def test_height_terms_polarised_mixed():
    """Four products x K terms share the gather kernel's complex sums (n_pol K <= 32 in FP32)."""
    prob = _jittered(72, radius=3, n_point=600, nside=4, polarised=True)
    out, info = _run(prob, fv.FV_MIXED, "terms")
    assert 2 <= info["height_terms"] <= 8 and out.shape[-1] == 4
    ref = oracle_vis(OracleProblem.from_workload(prob))
    for p in range(4):
        assert rel_l2(out[..., p], ref[..., p]) <= 2 * TOL[fv.FV_MIXED], p


def test_heights_auto_and_term_count():
    """Auto takes the terms for centimetre heights; the count grows with the heights and the accuracy."""
    flat = _jittered(73, z_sigma=0.01, n_chan=2, n_time=1, n_point=500, nside=0)
    _, i_flat = _run(flat, fv.FV_MIXED, "auto")
    assert i_flat["dims"] == 2 and i_flat["height_terms"] >= 1
    _, i_fp64 = _run(flat, fv.FV_FP64, "terms")
    assert i_fp64["height_terms"] > i_flat["height_terms"]           # eps 1e-11 vs 1e-6
    tall = _jittered(73, z_sigma=0.3, n_chan=2, n_time=1, n_point=500, nside=0)
    _, i_tall = _run(tall, fv.FV_MIXED, "terms")
    assert i_tall["height_terms"] > i_flat["height_terms"]
    # a coplanar array has no up axis: no terms whatever the option
    cop = _jittered(73, z_sigma=0.0, n_chan=2, n_time=1, n_point=500, nside=0)
    _, i_cop = _run(cop, fv.FV_MIXED, "terms")
    assert i_cop["dims"] == 2 and i_cop["height_terms"] == 0


def test_heights_grid_and_refusals():
    prob = _jittered(74, n_chan=2, n_time=1, n_point=500, nside=0)
    _, info = _run(prob, fv.FV_MIXED, "grid")
    assert info["dims"] == 3 and info["height_terms"] == 0
    # the terms are spread by the gather kernel only
    with pytest.raises(fv.FvError) as ei:
        _run(prob, fv.FV_MIXED, "terms", spread="scatter")
    assert ei.value.status == fv.FV_ERR_UNSUPPORTED
    # metre heights need more than 16 terms: refused when asked for, the grid in auto mode
    tall = _jittered(74, z_sigma=3.0, n_chan=2, n_time=1, n_point=500, nside=0)
    with pytest.raises(fv.FvError) as ei:
        _run(tall, fv.FV_FP64, "terms")
    assert ei.value.status == fv.FV_ERR_UNSUPPORTED
    _, i_auto = _run(tall, fv.FV_MIXED, "auto")
    assert i_auto["dims"] == 3 and i_auto["height_terms"] == 0
