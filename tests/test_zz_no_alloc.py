"""fv_execute_static: the entry point for callers that cannot allocate device
memory (a host whose own allocator owns the free HBM, a serving loop held to
a fixed HBM budget, a plug-in whose host forbids foreign allocations).  It
must give fv_execute's result, call after call, from the library's static
scratch, allocate nothing, and refuse plans whose scratch does not fit.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from oracle.oracle import OracleProblem, oracle_vis, rel_l2
from paper_2506_02130_gb300 import fv, workloads as W

pytestmark = pytest.mark.gpu

TOL = {fv.FV_FP64: 1e-9, fv.FV_MIXED: 2e-5}


def _plan(prob, precision, eps, transform="auto"):
    p = fv.Plan.from_problem(prob, precision=precision, eps=eps, transform=transform)
    p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
    return p


def _small_problem(seed):
    return W.config_hex127(seed=seed, n_chan=3, n_time=2, n_point=1200, nside=8, radius=2)


@pytest.mark.parametrize("transform", ["type3", "lattice"])
@pytest.mark.parametrize("precision,eps", [(fv.FV_MIXED, 1e-6), (fv.FV_FP64, 1e-11)])
def test_static_scratch_matches_fv_execute_twice(precision, eps, transform):
    torch = pytest.importorskip("torch")
    prob = _small_problem(21)
    cdt = torch.complex64 if precision == fv.FV_MIXED else torch.complex128
    # the static entry first, on a fresh plan that never allocated its own workspaces ...
    p = _plan(prob, precision, eps, transform)
    ws0 = p.info()["workspace_bytes"]
    outs = []
    for _ in range(2):
        out = torch.full(p.out_shape, float("nan"), dtype=cdt, device="cuda")
        fv.fv_execute_static(p.handle, out)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    assert p.info()["workspace_bytes"] == ws0
    # ... then fv_execute on a second plan built the same way
    q = _plan(prob, precision, eps, transform)
    ref = torch.empty(q.out_shape, dtype=cdt, device="cuda")
    fv.fv_execute(q.handle, ref)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    for got in outs:
        assert np.isfinite(got).all()
        assert rel_l2(got, ref) <= TOL[precision]
    p.close()
    q.close()


def test_static_call_allocates_no_device_memory():
    torch = pytest.importorskip("torch")
    prob = _small_problem(24)
    p = _plan(prob, fv.FV_MIXED, 1e-6, "type3")
    out = torch.empty(p.out_shape, dtype=torch.complex64, device="cuda")
    fv.fv_execute_static(p.handle, out)      # first call on the device: module load and address lookup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        fv.fv_execute_static(p.handle, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    p.close()


def test_static_scratch_large_then_small_plan_of_the_other_route():
    """The array keeps the previous call's contents: a large type-3 plan followed by a small lattice plan
    (and back) must each still match the direct sum."""
    torch = pytest.importorskip("torch")
    big = W.config_hex127(seed=25, n_chan=2, n_time=1, n_point=3000, nside=8, radius=4)
    small = W.config_hex127(seed=26, n_chan=1, n_time=2, n_point=200, nside=0, radius=2)
    small.ant_enu = W.hex_array(2)
    pb = _plan(big, fv.FV_MIXED, 1e-6, "type3")
    ps = _plan(small, fv.FV_MIXED, 1e-6, "lattice")
    assert ps.info()["transform"] == "lattice"
    refs = {id(pb): oracle_vis(OracleProblem.from_workload(big)),
            id(ps): oracle_vis(OracleProblem.from_workload(small))}
    for p in (pb, ps, pb, ps):
        out = torch.full(p.out_shape, float("nan"), dtype=torch.complex64, device="cuda")
        fv.fv_execute_static(p.handle, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel_l2(got, refs[id(p)]) <= 2e-5
    pb.close()
    ps.close()


def test_static_scratch_refuses_oversize_plans_and_host_buffers():
    torch = pytest.importorskip("torch")
    # 127 antennas at 200 MHz on the type-3 route: about 100 MB of per-slice scratch > 64 MiB
    prob = W.config_hex127(seed=22, n_chan=1, n_time=1, n_point=500, nside=0)
    prob.freqs_hz = np.array([200e6])
    prob.sky.flux = prob.sky.flux[:, :, :1]
    p = _plan(prob, fv.FV_MIXED, 1e-6, "type3")
    out = torch.zeros(p.out_shape, dtype=torch.complex64, device="cuda")
    with pytest.raises(fv.FvError) as ei:
        fv.fv_execute_static(p.handle, out)
    assert ei.value.status == fv.FV_ERR_UNSUPPORTED
    assert "static scratch" in str(ei.value)
    p.close()
    small = _plan(W.config_small(seed=23, n_src=200), fv.FV_MIXED, 1e-6)
    with pytest.raises(fv.FvError) as ei:
        fv.fv_execute_static(small.handle, np.zeros(small.out_shape, np.complex64))
    assert ei.value.status == fv.FV_ERR_ARG
    small.close()


@pytest.mark.parametrize("precision,eps,dtype", [(fv.FV_MIXED, 1e-6, "float32"), (fv.FV_FP64, 1e-11, "float64")])
def test_device_output_not_aligned_to_its_element_size_is_refused(precision, eps, dtype):
    # the kernels store a complex value with one 8- or 16-byte access, so an output that starts half an
    # element off is refused before anything is enqueued
    torch = pytest.importorskip("torch")
    prob = W.config_small(seed=24, n_src=200)
    p = _plan(prob, precision, eps)
    n = int(np.prod(p.out_shape)) * 2
    buf = torch.zeros(n + 1, dtype=getattr(torch, dtype), device="cuda")
    for call in (fv.fv_execute, fv.fv_execute_static):
        with pytest.raises(fv.FvError) as ei:
            call(p.handle, buf[1:])
        assert ei.value.status == fv.FV_ERR_ARG and "aligned" in str(ei.value)
    # the plan is unharmed: an aligned view of the same buffer works
    fv.fv_execute(p.handle, buf[:n])
    torch.cuda.synchronize()
    assert bool(torch.isfinite(buf[:n]).all())
    p.close()
