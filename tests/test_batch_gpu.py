"""Batches: slices of several different plans on shared lanes, plain and
replayed from a CUDA graph, give each plan's own fv_execute result; every
plan's output also matches the oracle."""
import numpy as np
import pytest

from oracle.oracle import OracleProblem, oracle_vis, rel_l2
from paper_2506_02130_gb300 import fv, workloads as W

pytestmark = pytest.mark.gpu


def _problems():
    return [
        (W.config_hex127(seed=31, n_chan=2, n_time=2, n_point=800, nside=8, radius=3), fv.FV_MIXED, 1e-6),
        (W.config_small(seed=32, n_src=600), fv.FV_FP64, 1e-10),
        (W.config_hex350_pol(seed=33, n_chan=2, n_time=1, n_point=300, nside=4, n_keep=None, radius=2), fv.FV_MIXED,
         1e-6),
        (W.config_hex127(seed=34, n_chan=1, n_time=3, n_point=500, nside=0, radius=2), fv.FV_FP64, 1e-11),
    ]


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_matches_each_plan_alone(use_graph):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    plans, outs, refs = [], [], []
    for prob, precision, eps in _problems():
        p = fv.Plan.from_problem(prob, precision=precision, eps=eps, stream=stream.cuda_stream)
        p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
        cdt = torch.complex64 if precision == fv.FV_MIXED else torch.complex128
        alone = torch.empty(p.out_shape, dtype=cdt, device=dev)
        p.run(alone)
        stream.synchronize()
        plans.append((p, prob, precision))
        refs.append(alone.cpu().numpy())
        outs.append(torch.full(p.out_shape, float("nan"), dtype=cdt, device=dev))
    b = fv.Batch(stream=stream.cuda_stream, n_lanes=3)
    for (p, prob, _), o in zip(plans, outs):
        b.add(p, o)
    for _ in range(2):           # the second execution replays the graph when use_graph
        b.execute(use_graph=use_graph)
        stream.synchronize()
        for (p, prob, precision), o, ref in zip(plans, outs, refs):
            got = o.cpu().numpy()
            tol = 2e-5 if precision == fv.FV_MIXED else 1e-9
            assert np.isfinite(got).all()
            assert rel_l2(got, ref) <= tol * 0.01
            assert rel_l2(got, oracle_vis(OracleProblem.from_workload(prob))) <= tol * (2 if prob.polarized else 1)
    assert b.workspace_bytes > 0
    b.close()
    for p, _, _ in plans:
        p.close()


def test_batch_partial_ranges_and_errors():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    prob = W.config_hex127(seed=35, n_chan=4, n_time=3, n_point=400, nside=0, radius=2)
    p = fv.Plan.from_problem(prob, precision=fv.FV_MIXED, eps=1e-6)
    p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
    full = p.run()
    out = torch.zeros(p.out_shape, dtype=torch.complex64, device=dev)
    b = fv.Batch(n_lanes=2)
    b.add(p, out, t_range=(1, 3), f_range=(2, 4))
    b.execute()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert rel_l2(got[2:4, 1:3], full[2:4, 1:3]) <= 1e-7
    assert np.all(got[:2] == 0) and np.all(got[:, 0] == 0)
    with pytest.raises(fv.FvError) as ei:
        b.add(p, out, t_range=(0, 9))
    assert ei.value.status == fv.FV_ERR_ARG
    with pytest.raises(fv.FvError) as ei:
        b.add(p, np.zeros(p.out_shape, np.complex64))
    assert ei.value.status == fv.FV_ERR_ARG
    b.close()
    p.close()


def test_batch_window_pieces_land_in_one_request_buffer():
    """fv_batch_add_range: pieces (one time, a block of channels) of a window
    of channels and times all land in one buffer shaped for the window."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    prob = W.config_hex127(seed=36, n_chan=5, n_time=4, n_point=300, nside=0, radius=2)
    p = fv.Plan.from_problem(prob, precision=fv.FV_FP64, eps=1e-10)
    p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
    full = p.run()
    f0, f1, t0, t1 = 1, 5, 1, 3
    win = torch.full((f1 - f0, t1 - t0, p.n_bl, p.n_pol), float("nan"), dtype=torch.complex128, device=dev)
    b = fv.Batch(n_lanes=3)
    b.add(p, win, t_range=(1, 2), f_range=(1, 3), window=(f0, t0, t1 - t0))
    b.add(p, win, t_range=(1, 2), f_range=(3, 5), window=(f0, t0, t1 - t0))
    b.add(p, win, t_range=(2, 3), f_range=(1, 5), window=(f0, t0, t1 - t0))
    b.execute(use_graph=True)
    torch.cuda.synchronize()
    got = win.cpu().numpy()
    assert np.isfinite(got).all()
    assert rel_l2(got, full[f0:f1, t0:t1]) <= 1e-12
    for bad in [dict(t_range=(0, 2), f_range=(1, 2)),      # t_lo before the window
                dict(t_range=(1, 4), f_range=(1, 2)),      # t_hi past the window
                dict(t_range=(1, 2), f_range=(0, 2))]:     # f_lo before the window
        with pytest.raises(fv.FvError) as ei:
            b.add(p, win, window=(f0, t0, t1 - t0), **bad)
        assert ei.value.status == fv.FV_ERR_ARG
    b.close()
    p.close()


def test_graph_is_captured_again_after_a_member_gets_a_new_sky():
    """A member plan's fv_set_sky after the graph was captured frees and replaces the buffers the graph
    points at (a larger sky, borrowed device flux at a new address): the next execution must capture again
    and give the new sky's visibilities, not replay kernels on freed memory."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    prob_a = W.config_hex127(seed=36, n_chan=2, n_time=2, n_point=300, nside=4, radius=3)
    prob_b = W.config_hex127(seed=37, n_chan=2, n_time=2, n_point=1500, nside=8, radius=3)
    # the same plan (array, channels, times) with another sky
    prob_b.ant_enu, prob_b.pairs, prob_b.lsts_rad = prob_a.ant_enu, prob_a.pairs, prob_a.lsts_rad
    assert np.array_equal(prob_b.freqs_hz, prob_a.freqs_hz)
    p = fv.Plan.from_problem(prob_a, precision=fv.FV_MIXED, eps=1e-6, stream=stream.cuda_stream)
    flux_a = torch.tensor(prob_a.sky.flux, dtype=torch.float32, device=dev)
    p.set_sky(prob_a.sky.ra, prob_a.sky.dec, flux_a)
    out = torch.full(p.out_shape, float("nan"), dtype=torch.complex64, device=dev)
    b = fv.Batch(stream=stream.cuda_stream, n_lanes=2)
    b.add(p, out)
    for _ in range(2):
        b.execute(use_graph=True)
    stream.synchronize()
    ref_a = oracle_vis(OracleProblem.from_workload(prob_a))
    assert rel_l2(out.cpu().numpy(), ref_a) <= 2e-5
    ws_a = b.workspace_bytes
    # a new, five times larger sky from a new device buffer; the old buffer is dropped
    flux_b = torch.tensor(prob_b.sky.flux, dtype=torch.float32, device=dev)
    p.set_sky(prob_b.sky.ra, prob_b.sky.dec, flux_b)
    del flux_a
    torch.cuda.empty_cache()
    out.fill_(float("nan"))
    for _ in range(2):
        b.execute(use_graph=True)
    stream.synchronize()
    alone = torch.empty(p.out_shape, dtype=torch.complex64, device=dev)
    p.run(alone)
    stream.synchronize()
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    assert rel_l2(got, alone.cpu().numpy()) <= 2e-7
    assert rel_l2(got, oracle_vis(OracleProblem.from_workload(prob_b))) <= 2e-5
    assert b.workspace_bytes >= ws_a
    b.close()
    p.close()
