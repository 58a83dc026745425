#!/usr/bin/env python
"""Visibility-path benchmark: visibilities/s of the type-3 NUFFT simulator.

Default workload (``--workload hex350``): 350-antenna coplanar hexagon (61,075
cross baselines), 256 channels at 100-200 MHz x 4 integrations, 886,432
polarised sources (100,000 power-law points + an nside-256 HEALPix diffuse
map), 2x2 Jones Airy beam of a 14 m dish, four polarisation products;
synthetic, seeded.  One step = fv_execute over all 1,024 (time, channel)
slices = 250,163,200 visibilities.  ``--workload hex127``: 127-antenna
hexagon with 5 cm height jitter, 64 channels x 10 integrations, 69,152
unpolarised sources, Gaussian beam (640 slices, 5,120,640 visibilities);
``batch`` and ``serve``: the ragged-slice batch and the request stream.

Default precision is the mixed path (FP32 spread/FFT/interp, FP64 phases,
eps 1e-6, accuracy gate 2e-5 relative L2); ``--precision fp64`` runs the FP64
path (eps 1e-11, gate 1e-9).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 direct-sum
oracle on the host cores instead (the reference arm for this path).
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target oracle CPU time for the baseline")
    ap.add_argument("--streams", type=int, default=0, help="execution streams per plan (0 = library default)")
    ap.add_argument("--spread", default="auto", choices=["auto", "gather", "scatter", "atomic", "tensor"])
    ap.add_argument("--fft-radix", type=int, default=0, choices=[0, 8, 16],
                    help="largest FFT stage radix of the timed plan (0: the library default)")
    ap.add_argument("--fp64-eps", type=float, default=1e-6,
                    help="tolerance of the plain FP64 comparison leg (its error is reported beside the mixed path's)")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip timing the plain FP64 path (one slice after another) beside the mixed path")
    ap.add_argument("--workload", default="hex350", choices=["hex350", "hex127", "batch", "serve"],
                    help="hex350: the 350-antenna polarised simulation, 256 channels x 4 times, 886,432 sources "
                         "(default); hex127: the 127-antenna, 64-channel, 10-time simulation; batch: 2,048 ragged "
                         "single-slice problems on shared lanes, replayed from a CUDA graph; serve: a Poisson "
                         "stream of requests over resident plans with continuous batching")
    ap.add_argument("--transform", default="type3", choices=["type3", "auto", "lattice", "basis"],
                    help="hex127: route of the timed plan (type3: the type-3 NUFFT of every slice)")
    ap.add_argument("--no-lattice-route", action="store_true",
                    help="hex127: skip timing the lattice route (Section 2.2.1 with height terms) beside it")
    ap.add_argument("--heights", default="auto", choices=["auto", "grid", "terms"],
                    help="up axis of a non-coplanar array on the type-3 route (the headline plan)")
    ap.add_argument("--no-heights-route", action="store_true",
                    help="skip the height-terms vs three-dimensional-grid comparison (non-coplanar arrays)")
    ap.add_argument("--no-tensor-leg", action="store_true",
                    help="skip the timing of the tensor-core spreading option")
    ap.add_argument("--no-basis-route", action="store_true",
                    help="hex127: skip timing the spectral-basis route (Appendix A) beside it")
    ap.add_argument("--basis-terms", type=int, default=0,
                    help="hex127: basis functions K of the spectral-basis route (0: chosen by the plan from "
                         "the sky's spectra against eps)")
    ap.add_argument("--channels", type=int, default=0,
                    help="hex350/hex127: keep this many channels across the same band (0 = all; a smaller case "
                         "of the same kernels for profiling, not a bench line)")
    ap.add_argument("--requests", type=int, default=200, help="serve: number of requests")
    ap.add_argument("--leg-requests", type=int, default=200,
                    help="hex350: requests of the serving leg run beside the headline")
    ap.add_argument("--no-serve-leg", action="store_true", help="hex350: skip the serving leg")
    ap.add_argument("--no-batch-leg", action="store_true", help="hex350: skip the batching leg")
    ap.add_argument("--rate", type=float, default=0.0,
                    help="serve: mean arrival rate (1/s); 0 = 70%% of the measured capacity for the request mix")
    ap.add_argument("--serve-scale", type=float, default=1.0, help="serve: sky size scale (1 = full skies)")
    ap.add_argument("--batch-slices", type=int, default=2048)
    ap.add_argument("--lanes", type=int, default=8, help="batch and serving execution lanes")
    ap.add_argument("--no-tune", action="store_true", help="batch: default choices instead of the autotuner")
    ap.add_argument("--batch-routes", default="auto",
                    help="batch: routes the autotuner may choose, comma separated (auto, type3)")
    return ap.parse_args()


def kernel_profile(fv, prob, precision, eps, stream, device, flux_dev, args, **plan_kw):
    """Per kernel class {ms, launches, bytes} of one step of a one-stream plan (fv_profile_enable): with
    one stream no two kernels overlap, so every CUDA-event pair times one kernel alone."""
    import torch
    p = fv.Plan.from_problem(prob, precision=precision, eps=eps, stream=stream.cuda_stream, device=device,
                             n_streams=1, spread=args.spread, fft_max_radix=args.fft_radix, **plan_kw)
    try:
        p.set_sky(prob.sky.ra, prob.sky.dec, flux_dev)
        o = torch.empty(p.out_shape, dtype=torch.complex64 if precision == fv.FV_MIXED else torch.complex128,
                        device=torch.device("cuda", device))
        p.run(o)                                          # warm-up (lazy workspaces, caches)
        torch.cuda.synchronize(device)
        fv.fv_profile_read(p.handle)                      # reset counters
        fv.fv_profile_enable(p.handle, True)
        p.run(o)
        torch.cuda.synchronize(device)
        prof = fv.fv_profile_read(p.handle)
        fv.fv_profile_enable(p.handle, False)
        return prof
    finally:
        p.close()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# the source files that define each kernel class of the type-3 route (plus the shared device header)
KERNEL_FILES = {"bin": ("fv_spread.cu", "fv_staged.cuh"), "prep": ("fv_spread.cu", "fv_staged.cuh"),
                "spread": ("fv_spread.cu", "fv_spread_ring.cu", "fv_staged.cuh"), "fft_x": ("fv_fft.cu",),
                "fft_y": ("fv_fft.cu",), "fft_z": ("fv_fft.cu",), "interp": ("fv_kernels.cu",),
                "scatter": ("fv_kernels.cu",)}


def kernel_source_hash(kernel_class):
    """Digest of the sources a kernel class is compiled from: a traffic figure taken from an ncu
    capture holds only while they are unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2506_02130_gb300", "csrc")
    for n in ("fv_internal.cuh",) + KERNEL_FILES.get(kernel_class, ()):
        with open(os.path.join(csrc, n), "rb") as f:
            h.update(n.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_class, precision):
    """DRAM bytes per launch of a type-3 kernel class from the committed ncu summary, if its sources
    are those the capture was taken with."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d["per_launch"][precision][kernel_class]
        if e.get("source_hash") != kernel_source_hash(kernel_class):
            return None
        return e["dram_bytes"]
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_reference(args, rank, world):
    """Reference arm: the FP64 direct-sum oracle on the host cores, on the same workload as our arm; each
    step is one (time, channel) slice (on the 350-antenna workload: its seeded 1% baseline subsample)."""
    if rank != 0:
        return
    import numpy as np
    from oracle.oracle import OracleProblem, oracle_vis, max_threads
    wl = SIM.get(args.workload, SIM["hex350"])
    name = args.workload if args.workload in SIM else "hex350"
    prob = sim_problem(name, 2 if name == "hex350" else 1)
    sampler = OracleSampler(prob, wl["oracle_bl"])
    pairs = prob.pairs if sampler.sel is None else prob.pairs[sampler.sel]
    n_pol = 4 if prob.polarized else 1
    nf, nt = len(prob.freqs_hz), len(prob.lsts_rad)
    slices = [(k % nf, (k * 7) % nt) for k in range(args.warmup + args.steps)]
    times = []
    for i, (f, t) in enumerate(slices):
        p = OracleProblem.from_workload(prob, pairs=pairs, freq_idx=[f], time_idx=[t])
        t0 = time.perf_counter()
        oracle_vis(p, "factored")
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = args.steps * len(pairs) * n_pol / total
    sub = "" if sampler.sel is None else (f" ({len(pairs)} seeded baselines of {len(prob.pairs)}; "
                                          "subsampled-rate: direct-sum cost is proportional to baselines)")
    line = {"metric": "visibilities/s at <=2e-5 rel err vs FP64 direct sum", "impl": "reference", "value": value,
            "unit": "visibilities/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "what": wl["what"],
                       "step": "one (time, channel) slice, FP64 direct sum" + sub},
            "cpu_baseline": {"value": value, "unit": "visibilities/s", "cores": max_threads(), "kind": "oracle",
                             "sample": f"{args.steps} timed slices of {nf * nt}, {len(pairs)} baselines" + sub},
            "e2e": {"value": value, "unit": "visibilities/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


BATCH_METRIC = "visibilities/s at <=2e-5 rel err vs FP64 direct sum"


def run_batch(args, rank, world, local, dist):
    """2,048 ragged single-slice problems (hexagons of 37-331 antennas, 1e3-5e5
    sources, eps 1e-6 on the mixed path or 1e-9 on the FP64 path) on shared
    lanes: autotuned plans, one batch, replayed from a CUDA graph."""
    import numpy as np
    import torch
    from paper_2506_02130_gb300 import autotune as AT, fv, workloads as W
    from oracle.oracle import OracleProblem, oracle_vis, rel_l2, max_threads
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t_setup = time.perf_counter()
    slices = W.config_batch(seed=4 + rank, n_slices=args.batch_slices)
    stream = torch.cuda.Stream(device=dev)
    tuner = AT.Autotuner(AT.cuda_timer(stream), routes=tuple(args.batch_routes.split(",")))
    t0 = time.perf_counter()
    if not args.no_tune:
        tuner.tune(slices, AT.key_of, AT.precision_of)
    tune_s = time.perf_counter() - t0

    # one flux buffer and one output buffer per precision; every plan borrows a view of them
    precs = [AT.precision_of(bs) for bs in slices]
    fdt = {fv.FV_MIXED: torch.float32, fv.FV_FP64: torch.float64}
    cdt = {fv.FV_MIXED: torch.complex64, fv.FV_FP64: torch.complex128}
    n_flux = {q: sum(bs.problem.sky.n_src for bs, pq in zip(slices, precs) if pq == q) for q in fdt}
    n_out = {q: sum(len(bs.problem.pairs) for bs, pq in zip(slices, precs) if pq == q) for q in fdt}
    flux_host = {q: torch.empty(max(n_flux[q], 1), dtype=fdt[q]).pin_memory() for q in fdt}
    flux_dev = {q: torch.empty(max(n_flux[q], 1), dtype=fdt[q], device=dev) for q in fdt}
    out_dev = {q: torch.empty(max(n_out[q], 1), dtype=cdt[q], device=dev) for q in fdt}
    out_host = {q: torch.empty(max(n_out[q], 1), dtype=cdt[q]).pin_memory() for q in fdt}
    fo = {q: 0 for q in fdt}
    oo = {q: 0 for q in fdt}
    plans, views = [], []
    choices = {}
    for bs, q in zip(slices, precs):
        prob = bs.problem
        ns, nb = prob.sky.n_src, len(prob.pairs)
        flux_host[q][fo[q]:fo[q] + ns] = torch.from_numpy(np.ascontiguousarray(prob.sky.flux[0, :, 0]))
        ch = tuner.choice(q, len(prob.ant_enu), ns)
        choices[AT.key_of(bs)] = ch
        p = fv.Plan.from_problem(prob, precision=q, eps=bs.nufft_eps, stream=stream.cuda_stream, device=local,
                                 n_streams=1, **ch.plan_kwargs())
        fview = flux_dev[q][fo[q]:fo[q] + ns].view(1, ns, 1)
        flux_dev[q][fo[q]:fo[q] + ns].copy_(flux_host[q][fo[q]:fo[q] + ns])
        p.set_sky(prob.sky.ra, prob.sky.dec, fview)
        v = out_dev[q][oo[q]:oo[q] + nb].view(p.out_shape)
        plans.append(p)
        views.append((q, oo[q], nb))
        fo[q] += ns
        oo[q] += nb
    b = fv.Batch(device=local, stream=stream.cuda_stream, n_lanes=args.lanes)
    for p, (q, o, nb) in zip(plans, views):
        b.add(p, out_dev[q][o:o + nb].view(p.out_shape))
    stream.synchronize()
    setup_s = time.perf_counter() - t_setup
    n_vis = sum(n_out.values())

    for _ in range(max(args.warmup, 1)):
        b.execute(use_graph=True)
    torch.cuda.synchronize(dev)
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    clocks.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        b.execute(use_graph=True)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    if dist:
        dist.barrier()
        t = torch.tensor([ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * n_vis * args.steps / (ms / 1e3)
    result = {q: out_dev[q].cpu().numpy() for q in fdt}

    # end to end: H2D of every slice's fluxes, the graph, D2H of every visibility (pinned buffers)
    h2d = sum(flux_host[q].numel() * flux_host[q].element_size() for q in fdt if n_flux[q])
    d2h = sum(out_host[q].numel() * out_host[q].element_size() for q in fdt if n_out[q])
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            for q in fdt:
                flux_dev[q].copy_(flux_host[q], non_blocking=True)
            b.execute(use_graph=True)
            for q in fdt:
                out_host[q].copy_(out_dev[q], non_blocking=True)
            stream.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * n_vis * args.steps / e2e_s, "unit": "visibilities/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * e2e_s / args.steps,
           "path": "pinned host fluxes -> device (one copy per precision), fv_batch_execute from the graph, "
                   "device visibilities -> pinned host"}

    # per-kernel times and launch counts: one plain (not captured) execution with kernel timing on
    for p in plans:
        fv.fv_profile_read(p.handle)
        fv.fv_profile_enable(p.handle, True)
    b.execute(use_graph=False)
    torch.cuda.synchronize(dev)
    prof, prof_by = {}, {"mixed": {}, "fp64": {}}
    for p, q in zip(plans, precs):
        for k, v in fv.fv_profile_read(p.handle).items():
            for tgt in (prof, prof_by["fp64" if q == fv.FV_FP64 else "mixed"]):
                a = tgt.setdefault(k, {"ms": 0.0, "launches": 0, "bytes": 0.0})
                a["ms"] += v["ms"]; a["launches"] += v["launches"]; a["bytes"] += v["bytes"]
        fv.fv_profile_enable(p.handle, False)
    ours = {k: v for k, v in prof.items() if k != "memset" and v["launches"] > 0}
    dom = max(ours, key=lambda k: ours[k]["ms"]) if ours else None
    peak, peak_kind = peaks()
    roof = None
    if dom:
        d = ours[dom]
        achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind, "traffic": None,
                "algorithmic_bytes_per_launch": d["bytes"] / d["launches"], "avg_launch_ms": d["ms"] / d["launches"],
                "share_of_kernel_time": d["ms"] / sum(v["ms"] for v in prof.values()),
                "timing": "CUDA events around each launch on its lane, one plain execution after the timed region "
                          "(lanes overlap, so per-class times add concurrent launches)"}
    gpu_launches = int(sum(v["launches"] for k, v in prof.items() if k != "memset")) * args.steps

    # the plain FP64 path, one slice per fv_execute, each slice alone (device time of that call)
    plain = None
    if not args.no_fp64_compare:
        tot = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for bs in slices:
            prob = bs.problem
            p = fv.Plan.from_problem(prob, precision=fv.FV_FP64, eps=bs.nufft_eps, stream=stream.cuda_stream,
                                     device=local, n_streams=1, transform="type3")
            p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
            o = torch.empty(p.out_shape, dtype=torch.complex128, device=dev)
            p.run(o)
            e0.record(stream)
            p.run(o)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1) / 1e3
            p.close()
        plain = {"value": world * n_vis / tot, "unit": "visibilities/s", "ms_per_step": 1e3 * tot,
                 "what": "every slice alone through fv_execute on an FP64 type-3 plan (upsampling 2, the "
                         "slice's transform tolerance), "
                         "sum of the calls' device times"}

    # oracle on 2% of the slices (at most 256 sampled baselines each): errors per path and the CPU rate
    cpu, errs = None, {"mixed": [], "fp64": []}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rng = np.random.default_rng(7)
        pick = rng.choice(len(slices), size=max(1, len(slices) // 50), replace=False)
        t_or, n_or = 0.0, 0
        for k in pick:
            bs, (q, o, nb) = slices[k], views[k]
            prob = bs.problem
            sel = np.sort(rng.choice(nb, size=min(nb, 256), replace=False))
            op = OracleProblem.from_workload(prob, pairs=prob.pairs[sel])
            t0 = time.perf_counter()
            ref = oracle_vis(op, "factored")[0, 0]
            t_or += time.perf_counter() - t0
            n_or += len(sel)
            got = result[q][o:o + nb][sel].reshape(ref.shape)
            errs[bs.precision].append(rel_l2(got, ref))
        cpu = {"value": n_or / t_or, "unit": "visibilities/s", "cores": max_threads(), "kind": "oracle",
               "sample": f"{len(pick)} of {len(slices)} slices, up to 256 seeded baselines each, all sources, "
                         f"FP64 antenna-factored direct sum", "seconds": t_or}
    err = {k: {"max": max(v), "n_slices": len(v)} for k, v in errs.items() if v}

    by_prec = {("fp64" if q == fv.FV_FP64 else "mixed"): {"slices": int(sum(1 for x in precs if x == q)),
                                                          "visibilities": int(n_out[q])} for q in fdt}
    line = {"metric": BATCH_METRIC, "value": value, "unit": "visibilities/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32/f64 (eps 1e-6 slices), f64 (eps 1e-9 slices)", "data": "synthetic",
            "config": {"workload": f"batch_{len(slices)}_ragged_slices_hex37-331_1e3-5e5src",
                       "slices": by_prec, "lanes": args.lanes, "graph": True, "autotuned": not args.no_tune,
                       "tune_seconds": tune_s, "setup_seconds": setup_s, "tuned_classes": len(tuner.table),
                       "choices": {k: dataclasses.asdict(v) for k, v in sorted(tuner.table.items())},
                       "vis_per_step": n_vis,
                       "l2": f"inputs larger than L2: {sum(n_flux.values())} sources and {n_vis} outputs per step",
                       "parallelism": f"{world} independent batches (one per GPU)"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": ck, "gpu_launches": gpu_launches,
            "rel_l2_vs_oracle_sample": err, "fp64_plain": plain,
            "kernels": {k: {"ms_per_step": v["ms"], "launches_per_step": v["launches"],
                            "GBps": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 else None}
                        for k, v in prof.items() if v["launches"] > 0},
            "kernel_ms_by_precision": {q: {k: v["ms"] for k, v in d.items() if v["launches"] > 0}
                                       for q, d in prof_by.items()},
            "routes": {"lattice_slices": sum(1 for p in plans if p.info()["transform"] == "lattice"),
                       "type3_slices": sum(1 for p in plans if p.info()["transform"] == "type3")}}
    b.close()
    for p in plans:
        p.close()
    return line


def run_serve(args, rank, world, local, dist):
    """Requests over three resident plans (37/127/350 antennas, 256 channels,
    20 times): Poisson arrivals, admission by free HBM, continuous batching."""
    import numpy as np
    import torch
    from paper_2506_02130_gb300 import fv, serve, workloads as W
    from oracle.oracle import OracleProblem, oracle_vis, rel_l2, max_threads
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    NF, NT = 256, 20
    t_setup = time.perf_counter()
    probs = W.serve_plans(seed=5 + rank, n_chan=NF, n_time=NT, scale=args.serve_scale)
    ex = serve.GpuExecutor(device=local, n_lanes=args.lanes)
    plans = {}
    for k, prob in probs.items():
        p = fv.Plan.from_problem(prob, precision=fv.FV_MIXED, eps=1e-6, stream=ex.stream.cuda_stream,
                                 device=local, n_streams=1)
        p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
        plans[k] = p
    torch.cuda.synchronize(dev)

    # calibration: GPU seconds of one slice of each plan (a tick of 16 channels at one time, after a warm-up)
    slice_s = {}
    for k, p in plans.items():
        r = serve.Request(-1, 0.0, k, (0, 16), (0, 1))
        buf = ex.alloc(p, r)
        for _ in range(2):
            dt = ex.wait(ex.submit([(p, buf, r, (0, 0, 16))]))
        slice_s[k] = dt / 16
    reqs_w = W.serve_requests(seed=5 + rank, n_requests=args.requests, rate_hz=1.0, n_chan=NF, n_time=NT)
    mean_cost = sum((r.f_range[1] - r.f_range[0]) * (r.t_range[1] - r.t_range[0]) * slice_s[r.kind]
                    for r in reqs_w) / len(reqs_w)
    capacity = 1.0 / mean_cost
    rate = args.rate if args.rate > 0 else 0.7 * capacity
    reqs_w = W.serve_requests(seed=5 + rank, n_requests=args.requests, rate_hz=rate, n_chan=NF, n_time=NT)
    reqs = [serve.Request(r.rid, r.arrival_s, r.kind, r.f_range, r.t_range) for r in reqs_w]
    free, total = torch.cuda.mem_get_info(dev)
    budget = int(max(free - (16 << 30), free // 2))
    setup_s = time.perf_counter() - t_setup

    # ~1% of the requests, at least two of each array, are checked against the oracle
    rs = np.random.default_rng(9)
    sample = set(rs.choice(len(reqs), size=max(1, len(reqs) // 100), replace=False).tolist())
    for k in plans:
        ids = [r.rid for r in reqs if r.kind == k]
        sample.update(rs.choice(ids, size=min(2, len(ids)), replace=False).tolist())
    kept = {}

    d2h = [0]

    def on_done(r, out, res):
        # every result comes back to the host (end to end); ~1% are kept for the oracle check
        host = out.cpu()
        d2h[0] += host.numel() * host.element_size()
        if r.rid in sample:
            kept[r.rid] = host.numpy()

    for p in plans.values():
        fv.fv_profile_read(p.handle)          # reset the launch counters
    srv = serve.Server(plans, ex, budget, slice_s, max_live=64, tick_s=0.02)
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    clocks.start()
    res = srv.run(reqs, on_done=on_done)
    ck = clocks.stop()
    summ = serve.summary(res, srv.stats)
    value = world * summ["vis_per_s"]
    launches = 0
    for p in plans.values():
        launches += sum(v["launches"] for k, v in fv.fv_profile_read(p.handle).items() if k != "memset")

    # the plain FP64 path: one slice per fv_execute on an FP64 plan of each array (device time per slice)
    plain = None
    if not args.no_fp64_compare:
        per = {}
        for k, prob in probs.items():
            sub = prob
            fl = np.ascontiguousarray(sub.sky.flux[:, :, :4], dtype=np.float64)
            p64 = fv.Plan.create(sub.freqs_hz[:4], sub.lsts_rad[:1], sub.latitude_rad, sub.beam, sub.beam_param,
                                 fv.FV_FP64, 1e-11, sub.polarized, stream=ex.stream.cuda_stream, device=local,
                                 n_streams=1, transform="type3")
            p64.set_array(sub.ant_enu, sub.pairs)
            p64.set_sky(sub.sky.ra, sub.sky.dec, fl)
            o = torch.empty(p64.out_shape, dtype=torch.complex128, device=dev)
            p64.run(o)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ex.stream)
            p64.run(o)
            e1.record(ex.stream)
            e1.synchronize()
            per[k] = e0.elapsed_time(e1) / 1e3 / 4            # 4 slices, one fv_execute each would cost no less
            p64.close()
        t_plain = sum((r.f_range[1] - r.f_range[0]) * (r.t_range[1] - r.t_range[0]) * per[r.kind] for r in reqs)
        plain = {"value": world * summ["visibilities"] / t_plain, "unit": "visibilities/s",
                 "seconds_per_slice": per,
                 "what": "the same requests' slices on FP64 type-3 plans (eps 1e-11, upsampling 2), device time per slice "
                         "measured on 4 channels of each array, summed over every slice with no queueing"}

    # oracle on ~1% of the requests (48 sampled baselines, every slice of the request)
    cpu, errs = None, []
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_or, n_or = 0.0, 0
        for rid in sorted(kept):
            r = reqs[rid]
            prob = probs[r.kind]
            nb = len(prob.pairs)
            sel = np.sort(np.random.default_rng(rid).choice(nb, size=min(nb, 48), replace=False))
            fi, ti = list(range(*r.f_range)), list(range(*r.t_range))
            # bounded: at most 8 channels x 4 times of the request (2 x 1 on the 350-antenna sky)
            fi, ti = (fi[:2], ti[:1]) if prob.sky.n_src > 500000 else (fi[:8], ti[:4])
            op = OracleProblem.from_workload(prob, pairs=prob.pairs[sel], freq_idx=fi, time_idx=ti)
            t0 = time.perf_counter()
            ref = oracle_vis(op)
            t_or += time.perf_counter() - t0
            n_or += ref.size
            got = kept[rid][:len(fi), :len(ti)][:, :, sel]
            errs.append({"rid": rid, "kind": r.kind, "rel_l2": rel_l2(got, ref)})
        if n_or:
            cpu = {"value": n_or / t_or, "unit": "visibilities/s", "cores": max_threads(), "kind": "oracle",
                   "sample": f"{len(kept)} of {len(reqs)} requests (at least 2 per array), 48 seeded baselines, "
                             f"up to 8 channels x 4 times each (2 x 1 on the 350-antenna sky), FP64 "
                             f"antenna-factored direct sum", "seconds": t_or}

    line = {"metric": "visibilities/s at <=2e-5 rel err vs FP64 direct sum; p50/p99 request latency",
            "value": value, "unit": "visibilities/s", "n_gpus": world, "steps": 1, "warmup": 2,
            "ms_per_step": 1e3 * summ["span_s"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/f64", "data": "synthetic",
            "config": {"workload": f"serve_{len(reqs)}_requests_hex37_hex127_hex350_256ch_20t",
                       "requests": len(reqs), "rate_hz": rate, "capacity_hz_estimate": capacity,
                       "slice_seconds": slice_s, "hbm_budget_bytes": budget, "lanes": args.lanes,
                       "tick_s": 0.02, "max_live": 64, "sky_scale": args.serve_scale, "setup_seconds": setup_s,
                       "n_src": {k: int(v.sky.n_src) for k, v in probs.items()},
                       "n_bl": {k: int(len(v.pairs)) for k, v in probs.items()},
                       "l2": "inputs larger than L2: resident skies of up to "
                             f"{max(v.sky.n_src for v in probs.values())} sources",
                       "parallelism": f"{world} independent servers (one per GPU)"},
            "serving": summ, "clocks": ck, "gpu_launches": int(launches), "cpu_baseline": cpu,
            "rel_l2_vs_oracle_sample": {"max": max((e["rel_l2"] for e in errs), default=None), "requests": errs},
            "fp64_plain": plain,
            "e2e": {"value": value, "unit": "visibilities/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": int(d2h[0]),
                    "path": "the served run itself: wall clock from the first arrival to the last completion, "
                            "every result copied to the host on completion; requests carry only windows of "
                            "resident plans, so no input bytes cross per request"}}
    ex.close()
    for p in plans.values():
        p.close()
    return line


# The simulation workloads: name in the JSON line, generator, route extras that apply
SIM = {
    "hex350": {"name": "hex350_pol_61075bl_256ch_4t_886432src", "oracle_bl": 611,
               "what": "350-antenna coplanar hexagon (61,075 cross baselines), 256 channels at 100-200 MHz x 4 "
                       "times, 100,000 polarised power-law points + nside-256 polarised diffuse map (886,432 "
                       "sources), 2x2 Jones Airy beam of a 14 m dish, four polarisation products"},
    "hex127": {"name": "hex127_8001bl_64ch_10t_69152src", "oracle_bl": 0,
               "what": "127-antenna hexagon with 5 cm height jitter (8,001 baselines, 3-D), 64 channels x 10 "
                       "times, 20,000 points + nside-64 diffuse map (69,152 sources), Gaussian beam"},
}


def sim_problem(name, seed, n_chan=0):
    """The workload's problem; n_chan > 0 keeps n_chan channels across the same band (a smaller case of
    the same per-slice kernels, for profiling)."""
    import numpy as np
    from paper_2506_02130_gb300 import workloads as W
    kw = {"n_chan": n_chan} if n_chan > 0 else {}
    if name == "hex350":
        return W.config_hex350_pol(seed=seed, dtype=np.float32, **kw)
    return W.config_hex127(seed=seed, **kw)


def sim_workload(args):
    """The workload's entry of SIM, renamed when --channels shrinks it."""
    wl = dict(SIM[args.workload])
    if args.channels > 0:
        wl["name"] = re.sub(r"_\d+ch_", "_%dch_" % args.channels, wl["name"])
        wl["what"] += "; reduced to %d channels across the same band" % args.channels
    return wl


class OracleSampler:
    """Relative L2 errors of several GPU outputs against the FP64 oracle on the same sampled slices
    (and, on large arrays, a seeded subsample of baselines), plus the oracle's own rate.

    Slices are taken in a seeded random order; each GPU output registers the slices it covers (copied
    to the host before its buffers are freed), and ``run`` computes the oracle slice by slice until its
    time budget is spent, accumulating every output's squared error per polarisation product."""

    def __init__(self, prob, n_bl_sample, n_keep=48, seed=123):
        import numpy as np
        self.prob = prob
        nf, nt, nb = len(prob.freqs_hz), len(prob.lsts_rad), len(prob.pairs)
        rng = np.random.default_rng(seed)
        self.order = [divmod(int(k), nt) for k in rng.permutation(nf * nt)[:n_keep]]
        self.sel = np.sort(rng.choice(nb, size=n_bl_sample, replace=False)) if 0 < n_bl_sample < nb else None
        self.got = {}

    def take(self, key, out, slices=None):
        """Copy the sampled slices of a GPU output [f][t][bl][pol] (torch tensor) to the host."""
        import torch
        sel = None if self.sel is None else torch.as_tensor(self.sel, device=out.device)
        d = {}
        for (f, t) in (slices if slices is not None else self.order):
            v = out[f, t] if sel is None else out[f, t][sel]
            d[(f, t)] = v.cpu().numpy()
        self.got[key] = d

    def run(self, target_s, extra=()):
        """Oracle on the sampled slices (then on the slices of `extra`) until target_s seconds pass."""
        import numpy as np
        from oracle.oracle import OracleProblem, oracle_vis, max_threads
        prob = self.prob
        pairs = prob.pairs if self.sel is None else prob.pairs[self.sel]
        acc = {k: [0.0, 0.0, None, None] for k in self.got}
        t_total, n_vis, done = 0.0, 0, 0
        todo = list(self.order) + [s for s in extra if s not in self.order]
        n_main = len(self.order)
        for i, (f, t) in enumerate(todo):
            # the sampled slices while the budget lasts (at least one), then the slices `extra` asks for
            if i < n_main and i > 0 and t_total >= target_s:
                continue
            op = OracleProblem.from_workload(prob, pairs=pairs, freq_idx=[f], time_idx=[t])
            t0 = time.perf_counter()
            ref = oracle_vis(op, "factored")[0, 0]
            t_total += time.perf_counter() - t0
            n_vis += ref.size
            done += 1
            for k, d in self.got.items():
                if (f, t) not in d:
                    continue
                got = d[(f, t)].reshape(ref.shape)
                e2 = (np.abs(got - ref) ** 2).sum(axis=0)
                r2 = (np.abs(ref) ** 2).sum(axis=0)
                a = acc[k]
                a[0] += float(e2.sum()); a[1] += float(r2.sum())
                a[2] = e2 if a[2] is None else a[2] + e2
                a[3] = r2 if a[3] is None else a[3] + r2
        err = {}
        for k, (e, r, ep, rp) in acc.items():
            if r > 0:
                err[k] = float(np.sqrt(e / r))
                if ep is not None and len(ep) > 1:
                    err[k + "_per_product"] = [float(np.sqrt(x / y)) for x, y in zip(ep, rp)]
        nb = len(pairs)
        cpu = {"value": n_vis / t_total if t_total > 0 else None, "unit": "visibilities/s",
               "cores": max_threads(), "kind": "oracle",
               "sample": f"{done} (time, channel) slices of {len(prob.freqs_hz) * len(prob.lsts_rad)}, "
                         + (f"{nb} seeded baselines of {len(prob.pairs)} (subsampled-rate: direct-sum cost is "
                            f"proportional to baselines x slices x sources)" if self.sel is not None
                            else f"all {nb} baselines")
                         + f", all {prob.sky.n_src} sources, FP64 antenna-factored direct sum",
               "seconds": t_total}
        return cpu, err


def timed_steps(run, stream, steps):
    """Device time (ms) of `steps` calls of run(), bracketed by CUDA events on `stream`."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        run()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def run_sim(args, rank, world, local, dist):
    """One whole simulation (every (time, channel) slice of the workload) per step."""
    import numpy as np
    import torch
    from paper_2506_02130_gb300 import fv
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = sim_workload(args)
    precision = fv.FV_MIXED if args.precision == "mixed" else fv.FV_FP64
    eps = 1e-6 if precision == fv.FV_MIXED else 1e-11
    t_setup = time.perf_counter()
    # each rank simulates its own independent problem (weak scaling)
    prob = sim_problem(args.workload, (2 if args.workload == "hex350" else 1) + rank, args.channels)
    nf, nt = len(prob.freqs_hz), len(prob.lsts_rad)
    sampler = OracleSampler(prob, wl["oracle_bl"])
    # a dedicated stream: the plan runs on it and the timing events are recorded on it
    stream = torch.cuda.Stream(device=dev)
    plan = fv.Plan.from_problem(prob, precision=precision, eps=eps, stream=stream.cuda_stream, device=local,
                                n_streams=args.streams, spread=args.spread, transform=args.transform,
                                fft_max_radix=args.fft_radix, heights=args.heights,
                                n_basis=args.basis_terms if args.transform == "basis" else 0)
    fdt = torch.float32 if precision == fv.FV_MIXED else torch.float64
    cdt = torch.complex64 if precision == fv.FV_MIXED else torch.complex128
    flux_dev = torch.tensor(prob.sky.flux, dtype=fdt, device=dev)
    plan.set_sky(prob.sky.ra, prob.sky.dec, flux_dev)
    info = plan.info()
    out = torch.empty(plan.out_shape, dtype=cdt, device=dev)
    n_vis = int(np.prod(plan.out_shape))
    setup_s = time.perf_counter() - t_setup

    for _ in range(args.warmup):
        plan.run(out)
    torch.cuda.synchronize(dev)

    # ---- timed region: K steps, device-resident inputs and outputs, no per-launch instrumentation
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)
    step_ms = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for k in range(args.steps):
        plan.run(out)
        ev[k + 1].record(stream)
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    if dist:
        dist.barrier()
    ms = ev[0].elapsed_time(ev[-1])
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    if dist:
        t = torch.tensor([ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * n_vis * args.steps / (ms / 1e3)
    sampler.take(args.precision, out)

    # ---- per-kernel times: one more step with CUDA events around every launch (event records between
    # launches would perturb the timed region above), on a one-stream copy of the plan so that no two
    # kernels overlap and each event pair brackets one kernel alone
    prof = kernel_profile(fv, prob, precision, eps, stream, local, flux_dev, args,
                          transform=args.transform, n_basis=args.basis_terms if args.transform == "basis" else 0)

    # ---- roofline of the dominant kernel class
    ours = {k: v for k, v in prof.items() if k != "memset" and v["launches"] > 0}
    dom = max(ours, key=lambda k: ours[k]["ms"]) if ours else None
    peak, peak_kind = peaks()
    roof = None
    if dom:
        d = ours[dom]
        achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
        tr = ncu_traffic(dom, f"{args.workload}_{args.precision}") if args.transform == "type3" else None
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": tr, "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
                "avg_launch_ms": d["ms"] / d["launches"],
                "share_of_kernel_time": d["ms"] / sum(v["ms"] for v in prof.values()),
                "timing": "CUDA events around each launch, one step of a one-stream copy of the plan after the "
                          "timed region (kernels do not overlap, so each event pair times one kernel alone)"}
        if dom == "spread":
            # the spreading's arithmetic: n_pol w^2 complex-by-real multiply-adds (4 flops) per visible source
            # (about half the sky), against the FP32 FMA peak of 152 SMs x 128 lanes x 2 flops at the
            # maximum SM clock
            w = info["kernel_width"]
            flops = 0.5 * prob.sky.n_src * plan.n_pol * w * w * 4.0 if plan else 0.0
            fp32_peak = 152 * 128 * 2 * 2.070e9 / 1e12
            useful = flops / (d["ms"] / d["launches"] / 1e3) / 1e12
            roof["secondary"] = {"bound": "alu", "achieved": useful, "peak": fp32_peak, "unit": "TFLOP/s",
                                 "frac": useful / fp32_peak,
                                 "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz",
                                 "what": "useful FP32 flops of the spreading (n_pol w^2 complex x real "
                                         "multiply-adds per visible source)"}
            roof["note"] = ("neither bound is reached: the spreading is bound by instruction issue and "
                            "shared-memory latency (a warp's lanes cover 8 x 8 cells, of which a source "
                            "reaches about a quarter); ncu figures in profiles/")
    gpu_launches = int(sum(v["launches"] for k, v in prof.items() if k != "memset")) * args.steps

    # ---- end to end through the C ABI with host buffers (pinned): set_sky copies the step's inputs in,
    # fv_execute copies the visibilities out
    e2e = None
    if not args.no_e2e:
        flux_host = torch.from_numpy(np.ascontiguousarray(prob.sky.flux, dtype=np.float32 if
                                                          precision == fv.FV_MIXED else np.float64)).pin_memory()
        out_host = torch.empty(plan.out_shape, dtype=cdt).pin_memory()
        ra = np.ascontiguousarray(prob.sky.ra); dec = np.ascontiguousarray(prob.sky.dec)
        h2d = ra.nbytes + dec.nbytes + flux_host.numel() * flux_host.element_size()
        d2h = out_host.numel() * out_host.element_size()
        fh = flux_host.numpy()
        plan.set_sky(ra, dec, fh)
        plan.run(out_host.numpy())
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            plan.set_sky(ra, dec, fh)                 # H2D of the step's inputs
            plan.run(out_host.numpy())                # compute + D2H of the result
        e2e_s = time.perf_counter() - t0
        if dist:
            t = torch.tensor([e2e_s], dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": world * n_vis * args.steps / e2e_s, "unit": "visibilities/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": 1e3 * e2e_s / args.steps}
        del flux_host, out_host
    plan.close()
    plan = None
    del out

    def route_leg(key, **kw):
        p = fv.Plan.from_problem(prob, precision=precision, eps=eps, stream=stream.cuda_stream, device=local,
                                 n_streams=args.streams, **kw)
        p.set_sky(prob.sky.ra, prob.sky.dec, flux_dev)
        o = torch.empty(p.out_shape, dtype=cdt, device=dev)
        for _ in range(args.warmup):
            p.run(o)
        torch.cuda.synchronize(dev)
        msr = timed_steps(lambda: p.run(o), stream, args.steps)
        sampler.take(key, o)
        li = p.info()
        p.close()
        del o
        return {"value": world * n_vis * args.steps / (msr / 1e3), "unit": "visibilities/s",
                "ms_per_step": msr / args.steps}, li

    # ---- the lattice route on the same workload (Section 2.2.1; heights, if any, by Chebyshev terms)
    lat_route = None
    if args.transform == "type3" and not args.no_lattice_route:
        lat_route, li = route_leg("lattice_route", transform="lattice")
        lat_route.update({"lattice_terms": li["lattice_terms"], "lattice_modes": li["lattice_modes"],
                          "lattice_grid": li["lattice_grid"],
                          "what": "same workload, plan with transform=lattice (type-1 transforms on the "
                                  "horizontal lattice, heights by Chebyshev terms)"})

    # ---- the up axis of a non-coplanar array on the type-3 route: Chebyshev height terms on a 2-D grid
    # against the third grid dimension (Section 2.2.2), same workload, both timed like the headline
    hts = None
    nonplanar = bool(np.any(prob.ant_enu[:, 2] != prob.ant_enu[0, 2]))
    if args.transform == "type3" and not args.no_heights_route and nonplanar:
        hts = {"what": "same workload on the type-3 route: heights=terms (K two-dimensional transforms of "
                       "c T_q(u), Bessel-weighted per target) against heights=grid (a three-dimensional grid)"}
        for key, h in (("heights_terms", "terms"), ("heights_grid", "grid")):
            try:
                leg, hi = route_leg(key, transform="type3", heights=h)
                leg.update({"dims": hi["dims"], "height_terms": hi["height_terms"], "nf1_max": hi["nf1_max"]})
            except fv.FvError as e:
                leg = {"unavailable": str(e)}
            hts[h] = leg
        if "ms_per_step" in hts["terms"] and "ms_per_step" in hts["grid"]:
            hts["speedup_terms_over_grid"] = hts["grid"]["ms_per_step"] / hts["terms"]["ms_per_step"]

    # ---- the optional tensor-core form of the gather spreading (FP32 two-dimensional grids), same workload
    tens = None
    if args.transform == "type3" and precision == fv.FV_MIXED and not args.no_tensor_leg:
        try:
            tens, ti = route_leg("tensor_spread", transform="type3", spread="tensor", heights=args.heights)
            tens.update({"spread": ti["spread"],
                         "what": "same workload with spread=tensor: each warp's 8 x 8 block of cells summed as "
                                 "m16n8k8 TF32 tensor-core products with a three-term split (an option, off by "
                                 "default; FP32 FMAs otherwise)"})
            if ti["spread"] != "tensor":
                tens = None                  # not applicable here (three-dimensional grid, FP64, ...)
        except fv.FvError as e:
            tens = {"unavailable": str(e)}

    # ---- the spectral-basis route (Appendix A; scalar skies only)
    bas_route = None
    if args.transform == "type3" and not args.no_basis_route and not prob.polarized:
        bas_route, bi = route_leg("basis_route", transform="basis", n_basis=args.basis_terms)
        bprof = kernel_profile(fv, prob, precision, eps, stream, local, flux_dev, args, transform="basis",
                               n_basis=args.basis_terms)
        bas_route.update({"basis_terms": bi["basis_terms"], "basis_terms_chosen_by_plan": args.basis_terms == 0,
                          "basis_fit_error": bi["basis_fit_error"], "grid": bi["basis_grid"],
                          "kernels_ms_per_step": {k: v["ms"] for k, v in bprof.items() if v["launches"] > 0},
                          "what": "same workload, plan with transform=basis: per time one transform per basis "
                                  "function of the band (Appendix A), expanded to the channels in the "
                                  "interpolation"})

    # ---- the plain FP64 path at equal accuracy: one slice after another on one stream (no batching, no
    # concurrent slices), at the tolerance whose error matches the mixed path's; on the 350-antenna
    # workload a seeded subset of channels (all times) keeps the leg short
    fp64 = None
    extra_slices = []
    if precision == fv.FV_MIXED and not args.no_fp64_compare:
        del flux_dev
        torch.cuda.empty_cache()
        ch = list(range(0, nf, 16)) if nf > 64 else list(range(nf))
        sub_flux = np.ascontiguousarray(prob.sky.flux[:, :, ch], dtype=np.float64)
        p64 = fv.Plan.create(prob.freqs_hz[ch], prob.lsts_rad, prob.latitude_rad, prob.beam, prob.beam_param,
                             fv.FV_FP64, args.fp64_eps, prob.polarized, stream=stream.cuda_stream, device=local,
                             n_streams=1, transform="type3")
        p64.set_array(prob.ant_enu, prob.pairs)
        f64dev = torch.from_numpy(sub_flux).to(dev)
        p64.set_sky(prob.sky.ra, prob.sky.dec, f64dev)
        o64 = torch.empty(p64.out_shape, dtype=torch.complex128, device=dev)
        p64.run(o64)
        torch.cuda.synchronize(dev)
        ms64 = timed_steps(lambda: p64.run(o64), stream, 3)
        n64 = int(np.prod(p64.out_shape))
        # sampled slices of the subset, mapped back to the workload's channel index
        rng = np.random.default_rng(321)
        picks = [(int(a), int(b)) for a, b in zip(rng.choice(len(ch), 2), rng.choice(nt, 2))]
        sel = None if sampler.sel is None else torch.as_tensor(sampler.sel, device=dev)
        sampler.got["fp64_plain"] = {(ch[a], b): (o64[a, b] if sel is None else o64[a, b][sel]).cpu().numpy()
                                     for a, b in picks}
        extra_slices = [(ch[a], b) for a, b in picks]
        fp64 = {"value": world * n64 * 3 / (ms64 / 1e3), "unit": "visibilities/s", "ms_per_step": ms64 / 3,
                "eps": args.fp64_eps, "steps": 3, "warmup": 1, "streams": 1, "channels": len(ch),
                "visibilities_per_step": n64, "kernel_width": p64.info()["kernel_width"],
                "what": "plain FP64 type-3 path, one slice after another on one stream, at the tolerance whose "
                        "error against the direct sum matches the mixed path's (error in "
                        "rel_l2_vs_oracle_sample.fp64_plain)"
                        + (f"; channels {ch[0]}, {ch[1]}, ... (every 16th) of the {nf}, all times"
                           if len(ch) < nf else "")}
        p64.close()
        del o64, f64dev

    # ---- CPU baseline (oracle) on a bounded sample, rank 0 at N=1; reports the GPU errors on it too
    cpu, err = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, err = sampler.run(args.cpu_seconds, extra_slices)

    # ---- the serving and batching patterns on this GPU, beside the headline (each a short run of its own)
    serving_leg = batch_leg = None
    if args.workload == "hex350" and not args.no_serve_leg:
        a2 = argparse.Namespace(**vars(args))
        a2.requests, a2.rate, a2.no_fp64_compare = args.leg_requests, 0.0, True
        sv = run_serve(a2, rank, world, local, dist)
        serving_leg = {"value": sv["value"], "unit": sv["unit"], "requests": sv["config"]["requests"],
                       "rate_hz": sv["config"]["rate_hz"], "capacity_hz_estimate": sv["config"]["capacity_hz_estimate"],
                       "p50_latency_s": sv["serving"]["p50_latency_s"], "p99_latency_s": sv["serving"]["p99_latency_s"],
                       "mean_latency_s": sv["serving"]["mean_latency_s"], "p50_queue_s": sv["serving"]["p50_queue_s"],
                       "rel_l2_vs_oracle_max": sv["rel_l2_vs_oracle_sample"]["max"],
                       "workload": sv["config"]["workload"], "seconds": sv["ms_per_step"] / 1e3,
                       "what": "Poisson stream of requests (blocks of 1-256 channels x 1-20 times of resident 37-, "
                               "127- and 350-antenna plans) at 70% of the measured capacity; continuous batching, "
                               "admission by free HBM; latency from arrival to the result on the host"}
        torch.cuda.empty_cache()
    if args.workload == "hex350" and not args.no_batch_leg:
        a2 = argparse.Namespace(**vars(args))
        a2.steps, a2.warmup, a2.no_fp64_compare = 3, 2, True
        bt = run_batch(a2, rank, world, local, dist)
        batch_leg = {"value": bt["value"], "unit": bt["unit"], "ms_per_step": bt["ms_per_step"], "steps": 3,
                     "slices": bt["config"]["slices"], "workload": bt["config"]["workload"],
                     "rel_l2_vs_oracle_sample": bt["rel_l2_vs_oracle_sample"], "routes": bt["routes"],
                     "tune_seconds": bt["config"]["tune_seconds"],
                     "what": "2,048 ragged single-slice problems (37-331 antennas, 1e3-5e5 sources, eps 1e-6 on the "
                             "mixed path or 1e-9 on the FP64 path), autotuned, on shared lanes replayed from one "
                             "CUDA graph; errors per path on 2% of the slices against the direct sum"}
        torch.cuda.empty_cache()

    lat = sorted(step_ms)
    line = {"metric": "visibilities/s at <=2e-5 rel err vs FP64 direct sum", "value": value,
            "unit": "visibilities/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/f64" if precision == fv.FV_MIXED else "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "what": wl["what"], "n_ant": int(len(prob.ant_enu)),
                       "n_bl": info["n_bl"], "n_unique_targets": info["n_unique"], "n_freq": nf, "n_time": nt,
                       "n_pol": 4 if prob.polarized else 1,
                       "n_src": int(prob.sky.n_src), "dims": info["dims"], "height_terms": info["height_terms"], "precision": args.precision,
                       "eps": eps, "kernel_width": info["kernel_width"], "upsampfac": info["upsampfac"],
                       "nf1_max": info["nf1_max"], "nf2_max": info["nf2_max"],
                       "streams": args.streams or (4 if args.transform == "basis" else 8),
                       "spread": info.get("spread", args.spread), "spread_requested": args.spread,
                       "transform": args.transform, "vis_per_step": n_vis,
                       "setup_seconds": setup_s,
                       "l2": "inputs larger than L2: a step streams every slice's grid through the reused "
                             f"workspaces (~{info['workspace_bytes'] / 1e6:.0f} MB) and reads "
                             f"{prob.sky.flux.size * (4 if precision == fv.FV_MIXED else 8) / 1e9:.2f} GB of "
                             "fluxes",
                       "parallelism": f"{world} independent problems (one per GPU)"},
            "step_latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                                "min": lat[0], "max": lat[-1]},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": ck, "gpu_launches": gpu_launches,
            "rel_l2_vs_oracle_sample": err, "fp64_plain_equal_accuracy": fp64, "lattice_route": lat_route,
            "heights_route": hts, "tensor_spread": tens,
            "basis_route": bas_route, "serving": serving_leg, "batching": batch_leg,
            "kernels": {k: {"ms_per_step": v["ms"], "launches_per_step": v["launches"],
                            "GBps": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 else None}
                        for k, v in prof.items() if v["launches"] > 0}}
    return line


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
        if dist:
            dist.destroy_process_group()
        return
    if args.workload in ("batch", "serve"):
        line = (run_batch if args.workload == "batch" else run_serve)(args, rank, world, local, dist)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    line = run_sim(args, rank, world, local, dist)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
