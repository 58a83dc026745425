"""The batched workload: ragged single-slice problems (hexagons of 37-331
antennas, eps 1e-6 on the mixed path and 1e-9 on the FP64 path) with
autotuned plans, one batch replayed from a CUDA graph.  Every slice matches
the oracle on sampled baselines within its path's tolerance, and the batch
gives the same result as each plan run alone."""
import numpy as np
import pytest

from oracle.oracle import OracleProblem, oracle_vis, rel_l2
from paper_2506_02130_gb300 import autotune as AT, fv, workloads as W

pytestmark = pytest.mark.gpu

TOL = {"mixed": 2e-5, "fp64": 1e-9}


def _run(slices, tuner, stream, dev, torch, lanes=4):
    plans, outs = [], []
    for bs in slices:
        q = AT.precision_of(bs)
        ch = tuner.choice(q, len(bs.problem.ant_enu), bs.problem.sky.n_src)
        p = fv.Plan.from_problem(bs.problem, precision=q, eps=bs.nufft_eps, stream=stream.cuda_stream, n_streams=1,
                                 **ch.plan_kwargs())
        p.set_sky(bs.problem.sky.ra, bs.problem.sky.dec, bs.problem.sky.flux)
        plans.append(p)
        outs.append(torch.full(p.out_shape, float("nan"), dtype=torch.complex128 if q == fv.FV_FP64
                               else torch.complex64, device=dev))
    b = fv.Batch(stream=stream.cuda_stream, n_lanes=lanes)
    for p, o in zip(plans, outs):
        b.add(p, o)
    return plans, outs, b


def test_ragged_batch_autotuned_graph_matches_oracle():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    slices = W.config_batch(seed=40, n_slices=24, n_src_range=(1000, 30000))
    tuner = AT.Autotuner(AT.cuda_timer(stream, reps=1, warmup=1))
    tuner.tune(slices, AT.key_of, AT.precision_of)
    assert tuner.table
    plans, outs, b = _run(slices, tuner, stream, dev, torch)
    for _ in range(2):
        b.execute(use_graph=True)
    stream.synchronize()
    rng = np.random.default_rng(0)
    for bs, p, o in zip(slices, plans, outs):
        got = o.cpu().numpy()[0, 0]
        assert np.isfinite(got).all()
        nb = len(bs.problem.pairs)
        sel = np.sort(rng.choice(nb, size=min(nb, 128), replace=False))
        ref = oracle_vis(OracleProblem.from_workload(bs.problem, pairs=bs.problem.pairs[sel]))[0, 0]
        err = rel_l2(got[sel], ref)
        assert err <= TOL[bs.precision], (bs.problem.name, bs.precision, err)
        # the same plan alone (equal up to the summation order of shared-memory atomics when the tuner
        # picked the scatter spreader)
        alone = p.run()
        assert rel_l2(got, alone[0, 0]) <= TOL[bs.precision] * 0.1
    b.close()
    for p in plans:
        p.close()


def _fp64_slices(seed):
    slices = [s for s in W.config_batch(seed=seed, n_slices=16, radii=(3, 10), n_src_range=(2000, 8000))
              if s.precision == "fp64"][:3]
    assert slices
    return slices


def test_fp64_upsampling_2_meets_the_gate_for_eps_1e9_slices():
    pytest.importorskip("torch")
    for bs in _fp64_slices(41):
        p = fv.Plan.from_problem(bs.problem, precision=fv.FV_FP64, eps=bs.nufft_eps, upsampfac=2.0)
        p.set_sky(bs.problem.sky.ra, bs.problem.sky.dec, bs.problem.sky.flux)
        got = p.run()[0, 0]
        nb = len(bs.problem.pairs)
        sel = np.arange(0, nb, max(1, nb // 200))
        ref = oracle_vis(OracleProblem.from_workload(bs.problem, pairs=bs.problem.pairs[sel]))[0, 0]
        assert rel_l2(got[sel], ref) <= 1e-9
        p.close()


def test_upsampling_1_25_refuses_a_tolerance_its_widest_kernel_misses_and_meets_a_looser_one():
    """At sigma 1.25 the transform tolerance 1e-10 needs a kernel wider than
    16 points: the plan refuses it (the tuner then skips the candidate); at
    1e-8 it fits and the error stays within a few eps."""
    pytest.importorskip("torch")
    bs = _fp64_slices(42)[0]
    with pytest.raises(fv.FvError) as ei:
        fv.Plan.from_problem(bs.problem, precision=fv.FV_FP64, eps=1e-10, upsampfac=1.25)
    assert ei.value.status == fv.FV_ERR_UNSUPPORTED
    p = fv.Plan.from_problem(bs.problem, precision=fv.FV_FP64, eps=1e-8, upsampfac=1.25)
    assert p.info()["kernel_width"] == 16
    p.set_sky(bs.problem.sky.ra, bs.problem.sky.dec, bs.problem.sky.flux)
    got = p.run()[0, 0]
    ref = oracle_vis(OracleProblem.from_workload(bs.problem))[0, 0]
    assert rel_l2(got, ref) <= 1e-7
    p.close()


def _large_slices(seed):
    """Slices of the batched workload at the top of its source range (3e5-5e5 sources), on the largest
    arrays (331 antennas among them), with both drawn tolerances."""
    pool = W.config_batch(seed=seed, n_slices=12, radii=(9, 10), n_src_range=(300000, 500000))
    fp64 = [s for s in pool if s.precision == "fp64"][:2]
    mixed = [s for s in pool if s.precision == "mixed"][:2]
    assert fp64 and mixed
    assert any(len(s.problem.ant_enu) == 331 for s in fp64 + mixed)
    return mixed + fp64


@pytest.mark.parametrize("route", ["batch", "type3"])
def test_large_sky_slices_of_the_batched_workload_match_the_oracle(route):
    """The spreading paths that only large skies reach (many candidate chunks per tile, many bin rows per
    tile at the low channel ratio): through the autotuned graph batch (whatever route the plans take),
    and forced onto the type-3 route (the tiled gather spreading)."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    slices = _large_slices(43)
    rng = np.random.default_rng(1)
    if route == "batch":
        tuner = AT.Autotuner(AT.cuda_timer(stream, reps=1, warmup=1))
        tuner.tune(slices, AT.key_of, AT.precision_of)
        plans, outs, b = _run(slices, tuner, stream, dev, torch)
        for _ in range(2):
            b.execute(use_graph=True)
        stream.synchronize()
        results = [o.cpu().numpy()[0, 0] for o in outs]
        b.close()
        for p in plans:
            p.close()
    else:
        results = []
        for bs in slices:
            q = AT.precision_of(bs)
            p = fv.Plan.from_problem(bs.problem, precision=q, eps=bs.nufft_eps, stream=stream.cuda_stream,
                                     transform="type3")
            p.set_sky(bs.problem.sky.ra, bs.problem.sky.dec, bs.problem.sky.flux)
            results.append(p.run()[0, 0])
            p.close()
    for bs, got in zip(slices, results):
        assert np.isfinite(got).all()
        nb = len(bs.problem.pairs)
        sel = np.sort(rng.choice(nb, size=min(nb, 96), replace=False))
        ref = oracle_vis(OracleProblem.from_workload(bs.problem, pairs=bs.problem.pairs[sel]))[0, 0]
        err = rel_l2(got[sel], ref)
        assert err <= TOL[bs.precision], (route, bs.problem.name, bs.problem.sky.n_src, bs.precision, err)
