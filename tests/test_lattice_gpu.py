"""The lattice route (Section 2.2.1, type-1 transform) against the oracle and
against the type-3 route, on the GPU through the C ABI."""
import numpy as np
import pytest

from oracle.oracle import OracleProblem, oracle_vis, rel_l2
from paper_2506_02130_gb300 import fv, workloads as W

pytestmark = pytest.mark.gpu

TOL = {fv.FV_FP64: 1e-9, fv.FV_MIXED: 2e-5}
EPS = {fv.FV_FP64: 1e-11, fv.FV_MIXED: 1e-6}


def _run(prob, precision, transform, **kw):
    p = fv.Plan.create(prob.freqs_hz, prob.lsts_rad, prob.latitude_rad, prob.beam, prob.beam_param, precision,
                       EPS[precision], prob.polarized, transform=transform, **kw)
    p.set_array(prob.ant_enu, prob.pairs)
    p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
    out = p.run()
    info = p.info()
    p.close()
    return out, info


def _coplanar(seed, n_chan=3, n_time=2, radius=3, n_point=700, nside=4):
    prob = W.config_hex127(seed=seed, n_chan=n_chan, n_time=n_time, n_point=n_point, nside=nside, radius=radius)
    prob.ant_enu = W.hex_array(radius)        # no height jitter: a coplanar lattice
    return prob


@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
def test_lattice_route_matches_oracle_and_type3(precision):
    prob = _coplanar(61)
    ref = oracle_vis(OracleProblem.from_workload(prob))
    lat, info = _run(prob, precision, "lattice")
    assert info["transform"] == "lattice" and info["lattice"]
    assert max(info["lattice_modes"]) <= 13            # |n_d| <= 2r = 6 on a radius-3 hexagon
    assert rel_l2(lat, ref) <= TOL[precision]
    t3, info3 = _run(prob, precision, "type3")
    assert info3["transform"] == "type3" and info3["lattice"]
    assert rel_l2(lat, t3) <= 2 * TOL[precision]


def test_auto_route_choice_and_forced_lattice_on_a_non_lattice():
    prob = _coplanar(62, n_chan=1, n_time=1)
    _, info = _run(prob, fv.FV_MIXED, "auto")
    assert info["transform"] == "lattice" and info["lattice_terms"] == 1
    jit = W.config_hex127(seed=62, n_chan=1, n_time=1, n_point=300, nside=0, radius=3)
    _, info = _run(jit, fv.FV_MIXED, "auto")          # heights of a few cm: a few Chebyshev terms
    assert info["transform"] == "lattice" and info["lattice_terms"] > 1
    rnd = W.config_hex127(seed=62, n_chan=1, n_time=1, n_point=300, nside=0, radius=3)
    rnd.ant_enu = rnd.ant_enu + np.random.default_rng(5).uniform(-1, 1, rnd.ant_enu.shape)
    _, info = _run(rnd, fv.FV_MIXED, "auto")
    assert info["transform"] == "type3" and not info["lattice"]
    with pytest.raises(fv.FvError) as ei:
        _run(rnd, fv.FV_MIXED, "lattice")
    assert ei.value.status == fv.FV_ERR_UNSUPPORTED


@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
def test_height_terms_on_a_jittered_lattice_match_oracle_and_type3(precision):
    """5 cm heights over 100-200 MHz: exp(-i a u) expanded in Chebyshev terms."""
    prob = W.config_hex127(seed=67, n_chan=4, n_time=2, n_point=800, nside=4, radius=4)
    out, info = _run(prob, precision, "lattice")
    assert info["lattice_terms"] > 1
    ref = oracle_vis(OracleProblem.from_workload(prob))
    assert rel_l2(out, ref) <= TOL[precision]
    t3, info3 = _run(prob, precision, "type3", heights="grid")
    assert info3["dims"] == 3
    assert rel_l2(out, t3) <= 2 * TOL[precision]


def test_height_terms_with_tall_antennas():
    """Heights of decimetres need many terms; the route still meets the FP64 gate."""
    prob = W.config_hex127(seed=68, n_chan=2, n_time=1, n_point=500, nside=0, radius=3)
    prob.ant_enu = W.hex_array(3)
    prob.ant_enu[:, 2] = np.random.default_rng(1).normal(0, 0.3, len(prob.ant_enu))
    out, info = _run(prob, fv.FV_FP64, "lattice")
    assert 8 <= info["lattice_terms"] <= 24
    ref = oracle_vis(OracleProblem.from_workload(prob))
    assert rel_l2(out, ref) <= 1e-9


@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
def test_lattice_route_polarised_airy(precision):
    prob = W.config_hex350_pol(seed=63, n_chan=2, n_time=1, n_point=400, nside=4, n_keep=None, radius=3)
    out, info = _run(prob, precision, "lattice")
    assert info["transform"] == "lattice"
    ref = oracle_vis(OracleProblem.from_workload(prob))
    for p in range(4):
        assert rel_l2(out[..., p], ref[..., p]) <= TOL[precision] * 2, p


@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
def test_lattice_route_on_a_lattice_sky_equals_numpy_fft2(precision):
    from tests._lattice import lattice_case
    L = lattice_case(N=16, G=5)
    p = fv.Plan.create(L["freqs"], L["lsts"], L["lat"], "uniform", (), precision, EPS[precision], False,
                       transform="lattice")
    p.set_array(L["ant"], L["pairs"])
    p.set_sky(L["ra"], L["dec"], L["flux"])
    out = p.run()[0, 0, :, 0]
    assert p.info()["transform"] == "lattice"
    p.close()
    assert rel_l2(out, L["expected"]) <= TOL[precision]


def test_lattice_route_large_hexagon_sampled_and_single_source():
    # 331-antenna hexagon (54,615 baselines), one slice, oracle on sampled baselines
    prob = _coplanar(64, n_chan=1, n_time=1, radius=10, n_point=3000, nside=8)
    out, info = _run(prob, fv.FV_MIXED, "auto")
    assert info["transform"] == "lattice"
    sel = np.sort(np.random.default_rng(0).choice(len(prob.pairs), 400, replace=False))
    ref = oracle_vis(OracleProblem.from_workload(prob, pairs=prob.pairs[sel]))
    assert rel_l2(out[:, :, sel], ref) <= 2e-5
    # one source: every visibility has modulus c, error within a few eps of it
    one = _coplanar(65, n_chan=1, n_time=1, radius=4, n_point=1, nside=0)
    v, _ = _run(one, fv.FV_FP64, "lattice")
    r = oracle_vis(OracleProblem.from_workload(one))
    assert np.abs(v - r).max() <= 1e-9 * np.abs(r).max()


def test_lattice_plans_in_a_batch_with_windows():
    torch = pytest.importorskip("torch")
    prob = _coplanar(66, n_chan=5, n_time=3, radius=4)
    p = fv.Plan.from_problem(prob, precision=fv.FV_MIXED, eps=1e-6, transform="lattice")
    p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
    full = p.run()
    win = torch.full((3, 2, p.n_bl, 1), float("nan"), dtype=torch.complex64, device="cuda")
    b = fv.Batch(n_lanes=2)
    b.add(p, win, t_range=(1, 3), f_range=(2, 5), window=(2, 1, 2))
    b.execute(use_graph=True)
    torch.cuda.synchronize()
    got = win.cpu().numpy()
    assert rel_l2(got, full[2:5, 1:3]) <= 1e-6
    b.close()
    p.close()


def test_fp64_lattice_borrowed_flux_rescaled_in_place():
    """A borrowed device flux rewritten in place between executions (here x4) gives the linear
    result on the FP64 lattice route."""
    torch = pytest.importorskip("torch")
    prob = _coplanar(69, n_chan=2, n_time=1)
    p = fv.Plan.from_problem(prob, precision=fv.FV_FP64, eps=1e-11, transform="lattice")
    flux = torch.tensor(prob.sky.flux, dtype=torch.float64, device="cuda")
    p.set_sky(prob.sky.ra, prob.sky.dec, flux)
    a = p.run()
    flux.mul_(4.0)
    torch.cuda.synchronize()
    b = p.run()
    assert rel_l2(b, 4.0 * a) <= 1e-12
    ref = oracle_vis(OracleProblem.from_workload(prob))
    assert rel_l2(a, ref) <= 1e-9
    p.close()


def test_auto_keeps_polarised_plans_with_many_sources_on_type3():
    """Four products: auto takes the lattice route only while 6 n_src K < n_src + t3 (the lattice spreading's
    global atomics contend for many sources); a few hundred sources stay on the lattice route."""
    few = W.config_hex350_pol(seed=64, n_chan=1, n_time=1, n_point=300, nside=0, n_keep=None, radius=3)
    _, info = _run(few, fv.FV_MIXED, "auto")
    assert info["transform"] == "lattice"
    many = W.config_hex350_pol(seed=64, n_chan=1, n_time=1, n_point=40000, nside=0, n_keep=None, radius=3)
    out, info = _run(many, fv.FV_MIXED, "auto")
    n_src, t3 = many.sky.n_src, info["nf1_max"][0] * info["nf1_max"][1]
    assert 6 * n_src >= n_src + t3 and info["transform"] == "type3"
    ref = oracle_vis(OracleProblem.from_workload(many))
    for p in range(4):
        assert rel_l2(out[..., p], ref[..., p]) <= 2 * TOL[fv.FV_MIXED], p
