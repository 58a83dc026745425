#!/usr/bin/env python
"""Visibility-path benchmark: visibilities/s of the type-3 NUFFT simulator.

Workload: 127-antenna hexagon (8,001 cross baselines, 5 cm height jitter, so
the transform is 3-D), 64 channels at 100-200 MHz, 10 integrations at 10.7 s,
69,152 sources (20,000 power-law points + a 49,152-pixel HEALPix diffuse map),
Gaussian beam; synthetic, seeded.  One step = fv_execute over all 640
(time, channel) slices = 5,120,640 visibilities.

Default precision is the mixed path (FP32 spread/FFT/interp, FP64 phases,
eps 1e-6, accuracy gate 2e-5 relative L2); ``--precision fp64`` runs the FP64
path (eps 1e-11, gate 1e-9).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 direct-sum
oracle on the host cores instead (the reference arm for this path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
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
    ap.add_argument("--spread", default="auto", choices=["auto", "gather", "scatter", "atomic"])
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip timing the plain FP64 path (one slice after another) beside the mixed path")
    return ap.parse_args()


def workload(seed):
    from paper_2506_02130_gb300 import workloads as W
    return W.config_hex127(seed=seed)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2506_02130_gb300", "csrc")
    for n in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, n), "rb") as f:
            h.update(n.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_class, precision):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current kernels."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_hash") != kernel_source_hash():
            return None
        return d["per_launch_bytes"][precision][kernel_class]
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


def oracle_sample(prob, target_s, gpu_outs=None):
    """Time the FP64 oracle (as it stands) on whole slices of the workload.

    Runs one slice, then as many more as fit in ``target_s`` seconds; returns
    vis/s, thread count, a description and, for every GPU output in the dict
    ``gpu_outs``, its relative L2 error on those slices.
    """
    import numpy as np
    from oracle.oracle import OracleProblem, oracle_vis, rel_l2, max_threads
    nf, nt = len(prob.freqs_hz), len(prob.lsts_rad)
    order = np.random.default_rng(123).permutation(nf * nt)
    gpu_outs = gpu_outs or {}
    done, t_total, refs = [], 0.0, []
    gots = {k: [] for k in gpu_outs}
    for k in order:
        f, t = divmod(int(k), nt)
        p = OracleProblem.from_workload(prob, freq_idx=[f], time_idx=[t])
        t0 = time.perf_counter()
        ref = oracle_vis(p, "factored")
        t_total += time.perf_counter() - t0
        done.append((f, t))
        refs.append(ref[0, 0])
        for k, v in gpu_outs.items():
            gots[k].append(v[f, t])
        if t_total >= target_s:
            break
    n_vis = len(done) * len(prob.pairs) * (4 if prob.polarized else 1)
    err = {k: rel_l2(np.array(v), np.array(refs)) for k, v in gots.items()}
    return {"value": n_vis / t_total, "unit": "visibilities/s", "cores": max_threads(), "kind": "oracle",
            "sample": f"{len(done)} of {nf * nt} (time, channel) slices, all {len(prob.pairs)} baselines and "
                      f"{prob.sky.n_src} sources, FP64 antenna-factored direct sum",
            "seconds": t_total}, err


def run_reference(args, rank, world):
    """Reference arm: the FP64 direct-sum oracle on the host cores."""
    if rank != 0:
        return
    prob = workload(1)
    n_bl = len(prob.pairs)
    from oracle.oracle import OracleProblem, oracle_vis, max_threads
    nf, nt = len(prob.freqs_hz), len(prob.lsts_rad)
    slices = [(k % nf, (k * 7) % nt) for k in range(args.warmup + args.steps)]
    times = []
    for i, (f, t) in enumerate(slices):
        p = OracleProblem.from_workload(prob, freq_idx=[f], time_idx=[t])
        t0 = time.perf_counter()
        oracle_vis(p, "factored")
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = args.steps * n_bl / total
    line = {"metric": "visibilities/s at <=2e-5 rel err vs FP64 direct sum", "impl": "reference", "value": value,
            "unit": "visibilities/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "hex127_8001bl_64ch_10t_69152src", "step": "one (time, channel) slice, "
                       "all baselines and sources, FP64 direct sum"},
            "cpu_baseline": {"value": value, "unit": "visibilities/s", "cores": max_threads(), "kind": "oracle",
                             "sample": f"{args.steps} timed slices of {nf * nt}, all {n_bl} baselines"},
            "e2e": {"value": value, "unit": "visibilities/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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

    import numpy as np
    import torch
    from paper_2506_02130_gb300 import fv
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    precision = fv.FV_MIXED if args.precision == "mixed" else fv.FV_FP64
    eps = 1e-6 if precision == fv.FV_MIXED else 1e-11
    prob = workload(1 + rank)             # each rank simulates its own independent problem (weak scaling)
    # a dedicated stream: the plan runs on it and the timing events are recorded on it
    stream = torch.cuda.Stream(device=dev)
    plan = fv.Plan.from_problem(prob, precision=precision, eps=eps, stream=stream.cuda_stream, device=local,
                                n_streams=args.streams, spread=args.spread)
    fdt = torch.float32 if precision == fv.FV_MIXED else torch.float64
    cdt = torch.complex64 if precision == fv.FV_MIXED else torch.complex128
    flux_dev = torch.tensor(prob.sky.flux, dtype=fdt, device=dev)
    plan.set_sky(prob.sky.ra, prob.sky.dec, flux_dev)
    info = plan.info()
    out = torch.empty(plan.out_shape, dtype=cdt, device=dev)
    n_vis = int(np.prod(plan.out_shape))

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
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        plan.run(out)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    if dist:
        t = torch.tensor([ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * n_vis * args.steps / (ms / 1e3)

    # ---- per-kernel times: one more step with CUDA events around every launch, each on the
    # stream it runs on (event records between launches would perturb the timed region above)
    fv.fv_profile_read(plan.handle)                       # reset counters
    fv.fv_profile_enable(plan.handle, True)
    plan.run(out)
    torch.cuda.synchronize(dev)
    prof = fv.fv_profile_read(plan.handle)
    fv.fv_profile_enable(plan.handle, False)
    prof_steps = 1

    # ---- roofline of the dominant kernel class
    ours = {k: v for k, v in prof.items() if k != "memset" and v["launches"] > 0}
    dom = max(ours, key=lambda k: ours[k]["ms"]) if ours else None
    peak, peak_kind = peaks()
    roof = None
    if dom:
        d = ours[dom]
        achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
        tr = ncu_traffic(dom, args.precision)
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": tr, "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
                "avg_launch_ms": d["ms"] / d["launches"],
                "share_of_kernel_time": d["ms"] / sum(v["ms"] for v in prof.values()),
                "timing": "CUDA events around each launch on its own stream, one profiled step after the timed region"}
    gpu_launches = int(sum(v["launches"] for k, v in prof.items() if k != "memset")) * args.steps // prof_steps

    # ---- end to end through the C ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        flux_host = torch.tensor(prob.sky.flux, dtype=fdt).pin_memory()
        out_host = torch.empty(plan.out_shape, dtype=cdt).pin_memory()
        ra = np.ascontiguousarray(prob.sky.ra); dec = np.ascontiguousarray(prob.sky.dec)
        h2d = ra.nbytes + dec.nbytes + flux_host.numel() * flux_host.element_size()
        d2h = out_host.numel() * out_host.element_size()
        fh = flux_host.numpy()
        for _ in range(1):
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

    # ---- the plain FP64 path (one slice after another, no batching) on the same workload
    fp64 = None
    outs = {args.precision: out.cpu().numpy()}
    if precision == fv.FV_MIXED and not args.no_fp64_compare:
        plan.close()
        p64 = fv.Plan.from_problem(prob, precision=fv.FV_FP64, eps=1e-11, stream=stream.cuda_stream, device=local)
        p64.set_sky(prob.sky.ra, prob.sky.dec, torch.tensor(prob.sky.flux, dtype=torch.float64, device=dev))
        o64 = torch.empty(p64.out_shape, dtype=torch.complex128, device=dev)
        p64.run(o64)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p64.run(o64)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = e0.elapsed_time(e1)
        fp64 = {"value": world * n_vis / (ms64 / 1e3), "unit": "visibilities/s", "ms_per_step": ms64,
                "eps": 1e-11, "steps": 1, "warmup": 1, "info": p64.info()}
        outs["fp64"] = o64.cpu().numpy()
        p64.close()
        plan = None

    # ---- CPU baseline (oracle) on a bounded sample, rank 0 at N=1; reports the GPU errors on it too
    cpu, err = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, err = oracle_sample(prob, args.cpu_seconds, outs)

    line = {"metric": "visibilities/s at <=2e-5 rel err vs FP64 direct sum", "value": value,
            "unit": "visibilities/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/f64" if precision == fv.FV_MIXED else "f64", "data": "synthetic",
            "config": {"workload": "hex127_8001bl_64ch_10t_69152src", "n_ant": 127, "n_bl": info["n_bl"],
                       "n_unique_targets": info["n_unique"], "n_freq": 64, "n_time": 10,
                       "n_src": int(prob.sky.n_src), "dims": info["dims"], "precision": args.precision,
                       "eps": eps, "kernel_width": info["kernel_width"], "upsampfac": info["upsampfac"],
                       "nf1_max": info["nf1_max"], "nf2_max": info["nf2_max"], "streams": args.streams or 4,
                       "spread": args.spread,
                       "vis_per_step": n_vis,
                       "l2": "inputs larger than L2: a step streams the 640 slices' grids "
                             f"(~{info['workspace_bytes'] / 1e6:.0f} MB workspace reused per slice)",
                       "parallelism": f"{world} independent problems (one per GPU)"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": ck, "gpu_launches": gpu_launches,
            "rel_l2_vs_oracle_sample": err, "fp64_plain": fp64,
            "kernels": {k: {"ms_per_step": v["ms"] / prof_steps, "launches_per_step": v["launches"] / prof_steps,
                            "GBps": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 else None}
                        for k, v in prof.items() if v["launches"] > 0}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if plan is not None:
        plan.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
