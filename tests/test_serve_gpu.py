"""Serving on the GPU: requests over resident plans, admitted by memory and
batched continuously.  Each request's result is the same alone and in the
mix, and matches the oracle on sampled baselines."""
import numpy as np
import pytest

from oracle.oracle import OracleProblem, oracle_vis, rel_l2
from paper_2506_02130_gb300 import fv, serve, workloads as W

pytestmark = pytest.mark.gpu

NF, NT = 12, 4


def _setup(torch):
    ex = serve.GpuExecutor(device=0, n_lanes=4)
    probs = W.serve_plans(seed=51, n_chan=NF, n_time=NT, scale=0.03)
    plans = {}
    for k, prob in probs.items():
        p = fv.Plan.from_problem(prob, precision=fv.FV_MIXED, eps=1e-6, stream=ex.stream.cuda_stream, n_streams=1)
        p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
        plans[k] = p
    return ex, probs, plans


def _requests():
    rs = W.serve_requests(seed=52, n_requests=14, rate_hz=2000.0, n_chan=NF, n_time=NT)
    return [serve.Request(r.rid, r.arrival_s, r.kind, r.f_range, r.t_range) for r in rs]


def test_each_request_same_alone_and_in_the_mix_and_matches_oracle():
    torch = pytest.importorskip("torch")
    ex, probs, plans = _setup(torch)
    slice_s = {k: 2e-4 for k in plans}
    reqs = _requests()
    mixed = {}

    def keep(r, out, res):
        mixed[r.rid] = out.cpu().numpy()

    srv = serve.Server(plans, ex, hbm_budget=1 << 30, slice_s=slice_s, tick_s=2e-4)
    res = srv.run(reqs, on_done=keep)
    assert all(r.status == "ok" for r in res)
    assert srv.stats.max_live > 1                  # requests overlapped on the device
    assert max(srv.stats.tick_sizes) > 1           # ticks mixed pieces of several requests
    for r in reqs:
        alone = {}
        srv1 = serve.Server(plans, ex, hbm_budget=1 << 30, slice_s={k: 1.0 for k in plans}, tick_s=1.0)
        srv1.run([serve.Request(r.rid, 0.0, r.kind, r.f_range, r.t_range)],
                 on_done=lambda q, out, res: alone.__setitem__(q.rid, out.cpu().numpy()))
        a, m = alone[r.rid], mixed[r.rid]
        assert np.isfinite(m).all()
        assert rel_l2(m, a) <= 2e-5 * 1e-2
        prob = probs[r.kind]
        nb = len(prob.pairs)
        sel = np.sort(np.random.default_rng(r.rid).choice(nb, size=min(nb, 48), replace=False))
        op = OracleProblem.from_workload(prob, pairs=prob.pairs[sel], freq_idx=list(range(*r.f_range)),
                                         time_idx=list(range(*r.t_range)))
        ref = oracle_vis(op)
        tol = 2e-5 * (2 if prob.polarized else 1)
        assert rel_l2(m[:, :, sel], ref) <= tol, (r.rid, r.kind)
    ex.close()
    for p in plans.values():
        p.close()


def test_memory_budget_holds_requests_back():
    torch = pytest.importorskip("torch")
    ex, probs, plans = _setup(torch)
    reqs = _requests()
    srv0 = serve.Server(plans, ex, hbm_budget=1 << 40, slice_s={k: 1e-4 for k in plans})
    biggest = max(srv0.out_bytes(r) for r in reqs)
    srv = serve.Server(plans, ex, hbm_budget=biggest, slice_s={k: 1e-4 for k in plans}, tick_s=1e-3)
    res = srv.run(reqs)
    assert all(r.status == "ok" for r in res)
    assert srv.stats.peak_reserved <= biggest
    s = serve.summary(res, srv.stats)
    assert s["served"] == len(reqs) and s["p99_latency_s"] >= s["p50_latency_s"] > 0
    ex.close()
    for p in plans.values():
        p.close()
