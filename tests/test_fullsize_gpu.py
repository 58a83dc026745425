"""Full-size workloads on the GPU, in the launch configuration bench.py times
(a dedicated stream, device-resident flux, the default stream count),
checked against the FP64 oracle on sampled outputs it computes one by one.

* 127-antenna hexagon (8,001 baselines, 3-D), 64 channels x 10 times,
  69,152 sources: the type-3 route on the mixed and FP64 paths, the lattice
  route and the spectral-basis route (12 basis functions) on the mixed path,
  three whole sampled slices each, against the direct sum.
* 350-antenna hexagon (61,075 baselines), 256 channels x 4 times, 886,432
  polarised sources, Airy Jones beam, mixed path: 611 sampled baselines
  (1%) of two sampled slices, all four products.
"""
import numpy as np
import pytest

from oracle.oracle import OracleProblem, oracle_vis, rel_l2
from paper_2506_02130_gb300 import fv, workloads as W

pytestmark = pytest.mark.gpu


def _run_on_stream(prob, precision, eps, flux_dtype, **plan_kw):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    plan = fv.Plan.from_problem(prob, precision=precision, eps=eps, stream=stream.cuda_stream, **plan_kw)
    flux = torch.tensor(prob.sky.flux, dtype=flux_dtype, device=dev)
    plan.set_sky(prob.sky.ra, prob.sky.dec, flux)
    cdt = torch.complex64 if precision == fv.FV_MIXED else torch.complex128
    out = torch.empty(plan.out_shape, dtype=cdt, device=dev)
    plan.run(out)
    stream.synchronize()
    return plan, out


# the routes bench.py times on this workload: the type-3 headline (both paths), the lattice route and the
# spectral-basis route with its 12 basis functions, each gated against the direct sum itself
@pytest.mark.parametrize("precision,eps,tol,route", [(fv.FV_MIXED, 1e-6, 2e-5, {"transform": "type3"}),
                                                     (fv.FV_FP64, 1e-11, 1e-9, {"transform": "type3"}),
                                                     (fv.FV_MIXED, 1e-6, 2e-5, {"transform": "lattice"}),
                                                     (fv.FV_MIXED, 1e-6, 2e-5, {"transform": "basis", "n_basis": 12}),
                                                     (fv.FV_MIXED, 1e-6, 2e-5, {"transform": "basis", "n_basis": 0}),
                                                     (fv.FV_FP64, 1e-11, 1e-9, {"transform": "basis", "n_basis": 16})],
                         ids=["type3-mixed", "type3-fp64", "lattice-mixed", "basis12-mixed", "basisauto-mixed",
                              "basis16-fp64"])
def test_hex127_full_size_sampled_slices(precision, eps, tol, route):
    torch = pytest.importorskip("torch")
    prob = W.config_hex127(seed=1)
    plan, out = _run_on_stream(prob, precision, eps, torch.float32 if precision == fv.FV_MIXED else torch.float64,
                               **route)
    assert plan.info()["transform"] == route["transform"]
    rng = np.random.default_rng(7)
    nf, nt = len(prob.freqs_hz), len(prob.lsts_rad)
    for k in rng.choice(nf * nt, 3, replace=False):
        f, t = divmod(int(k), nt)
        ref = oracle_vis(OracleProblem.from_workload(prob, freq_idx=[f], time_idx=[t]), "factored")[0, 0]
        got = out[f, t].cpu().numpy()
        assert rel_l2(got, ref) <= tol, (f, t, rel_l2(got, ref))
    plan.close()


def test_hex350_polarised_full_size_sampled_baselines():
    torch = pytest.importorskip("torch")
    prob = W.config_hex350_pol(seed=2, dtype=np.float32)
    assert prob.sky.n_src == 886432 and len(prob.pairs) == 61075
    plan, out = _run_on_stream(prob, fv.FV_MIXED, 1e-6, torch.float32)
    rng = np.random.default_rng(8)
    sel = np.sort(rng.choice(len(prob.pairs), 611, replace=False))
    nf, nt = len(prob.freqs_hz), len(prob.lsts_rad)
    for k in rng.choice(nf * nt, 2, replace=False):
        f, t = divmod(int(k), nt)
        ref = oracle_vis(OracleProblem.from_workload(prob, pairs=prob.pairs[sel], freq_idx=[f], time_idx=[t]),
                         "factored")[0, 0]
        got = out[f, t][torch.as_tensor(sel, device=out.device)].cpu().numpy()
        for p in range(4):
            assert rel_l2(got[:, p], ref[:, p]) <= 2e-5, (f, t, p, rel_l2(got[:, p], ref[:, p]))
    plan.close()
