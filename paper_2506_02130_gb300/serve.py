"""Serving: a request loop with continuous batching over resident plans.

The paper runs a simulation's (time, frequency) work as independent pieces
in parallel processes that share the read-only sky and beam (Section 5.4).
A GPU server does the same across requests: each request names a resident
plan (an array and a sky, with the plan's band of channels and grid of
times) and a window of channels and times.  The server

  * admits arrived requests in arrival order while their output buffers fit
    in the HBM budget and a slot is free (admission by free memory);
  * keeps every plan, its sky and its tables resident, so a request costs
    only its slices and its output buffer;
  * runs ticks: each tick takes a bounded piece of work from every admitted
    request (one time, a block of channels, sized by the measured cost of a
    slice of that plan so that a tick lasts about ``tick_s`` seconds of GPU
    time) and executes all pieces as one batch on shared lanes
    (fv_batch_add_range writes each piece into its request's buffer);
  * keeps two ticks in flight, so the host builds the next tick while the
    GPU runs the current one, and requests that arrive meanwhile join at the
    next tick: their work overlaps on the device with that of requests
    already running;
  * reports each request's latency (completion minus arrival), its queueing
    delay, and the throughput in visibilities per second.

A request's result does not depend on what else is in the tick: every slice
is computed by the same kernels from the same plan, independently of the
other slices.  The executor is pluggable so that the scheduling logic can be
tested on the host.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field


@dataclass
class Request:
    rid: int
    arrival_s: float                 # offset from the start of the stream
    kind: str                        # name of a resident plan
    f_range: tuple                   # [f_lo, f_hi) channels of that plan
    t_range: tuple                   # [t_lo, t_hi) times of that plan

    @property
    def n_slices(self) -> int:
        return (self.f_range[1] - self.f_range[0]) * (self.t_range[1] - self.t_range[0])


@dataclass
class Result:
    rid: int
    kind: str
    arrival_s: float
    admitted_s: float
    finished_s: float
    n_vis: int
    status: str = "ok"

    @property
    def latency_s(self) -> float:
        return self.finished_s - self.arrival_s


@dataclass
class _Live:
    req: Request
    out: object
    nbytes: int
    todo: collections.deque          # pieces (t, f_lo, f_hi) not yet submitted
    in_flight: int = 0               # submitted pieces whose tick has not finished
    admitted_s: float = 0.0


@dataclass
class Stats:
    ticks: int = 0
    pieces: int = 0
    max_live: int = 0
    peak_reserved: int = 0
    rejected: int = 0
    gpu_s: float = 0.0
    tick_sizes: list = field(default_factory=list)


class Server:
    """Continuous batching over resident plans.

    plans:       {kind: plan} (each with n_bl, n_pol, n_freq, n_time, precision)
    executor:    see GpuExecutor
    hbm_budget:  bytes of request output buffers that may be held at once
    slice_s:     {kind: estimated GPU seconds of one slice}
    """

    def __init__(self, plans: dict, executor, hbm_budget: int, slice_s: dict, max_live: int = 64,
                 tick_s: float = 0.02, depth: int = 2):
        self.plans = plans
        self.ex = executor
        self.budget = int(hbm_budget)
        self.slice_s = dict(slice_s)
        self.max_live = max_live
        self.tick_s = tick_s
        self.depth = depth
        self.stats = Stats()

    def out_bytes(self, r: Request) -> int:
        p = self.plans[r.kind]
        return r.n_slices * p.n_bl * p.n_pol * self.ex.elem_bytes(p)

    @staticmethod
    def pieces(r: Request) -> collections.deque:
        """All of the request's slices as (t, f_lo, f_hi) rows, time-major."""
        return collections.deque((t, r.f_range[0], r.f_range[1]) for t in range(*r.t_range))

    def _take(self, lv: _Live, share_s: float):
        """Next piece of lv's work worth about share_s seconds: part of one time's channel row."""
        t, f0, f1 = lv.todo[0]
        k = max(1, min(f1 - f0, int(share_s / max(self.slice_s[lv.req.kind], 1e-9))))
        if k == f1 - f0:
            lv.todo.popleft()
        else:
            lv.todo[0] = (t, f0 + k, f1)
        return (t, f0, f0 + k)

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep, on_done=None) -> list:
        """Serve `requests` (sorted by arrival); returns one Result per request."""
        queue = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        live: list[_Live] = []
        reserved = 0
        ticks = collections.deque()         # (token, [(live, piece), ...])
        results = []
        t0 = clock()
        now = lambda: clock() - t0

        def finish(lv, status="ok"):
            nonlocal reserved
            res = Result(lv.req.rid, lv.req.kind, lv.req.arrival_s, lv.admitted_s, now(),
                         lv.req.n_slices * self.plans[lv.req.kind].n_bl * self.plans[lv.req.kind].n_pol, status)
            results.append(res)
            if on_done is not None:
                on_done(lv.req, lv.out, res)
            self.ex.free(lv.out)
            reserved -= lv.nbytes

        while queue or live or ticks:
            # admission: arrived requests, in order, while their buffers fit and a slot is free
            while queue and queue[0].arrival_s <= now() and len(live) < self.max_live:
                r = queue[0]
                need = self.out_bytes(r)
                if need > self.budget:
                    queue.popleft()
                    self.stats.rejected += 1
                    results.append(Result(r.rid, r.kind, r.arrival_s, now(), now(), 0, "rejected: exceeds budget"))
                    continue
                if reserved + need > self.budget:
                    break
                queue.popleft()
                out = self.ex.alloc(self.plans[r.kind], r)
                reserved += need
                live.append(_Live(r, out, need, self.pieces(r), 0, now()))
            self.stats.max_live = max(self.stats.max_live, len(live))
            self.stats.peak_reserved = max(self.stats.peak_reserved, reserved)

            # build and submit ticks until `depth` are in flight
            while len(ticks) < self.depth:
                ready = [lv for lv in live if lv.todo]
                if not ready:
                    break
                share = self.tick_s / len(ready)
                work = []
                for lv in ready:
                    pc = self._take(lv, share)
                    lv.in_flight += 1
                    work.append((lv, pc))
                token = self.ex.submit([(self.plans[lv.req.kind], lv.out, lv.req, pc) for lv, pc in work])
                ticks.append((token, work))
                self.stats.ticks += 1
                self.stats.pieces += len(work)
                self.stats.tick_sizes.append(len(work))

            if ticks:
                token, work = ticks.popleft()
                self.stats.gpu_s += self.ex.wait(token)
                for lv, _ in work:
                    lv.in_flight -= 1
                done = [lv for lv in live if not lv.todo and lv.in_flight == 0]
                for lv in done:
                    live.remove(lv)
                    finish(lv)
            elif queue:
                wait = queue[0].arrival_s - now()
                if wait > 0:
                    sleep(min(wait, 0.05))
        return sorted(results, key=lambda r: r.rid)


def percentile(xs, q: float) -> float:
    """q-th percentile (0-100) by linear interpolation between order statistics."""
    if not xs:
        return math.nan
    s = sorted(xs)
    pos = (len(s) - 1) * q / 100.0
    lo = int(math.floor(pos))
    hi = min(lo + 1, len(s) - 1)
    return s[lo] + (s[hi] - s[lo]) * (pos - lo)


def summary(results, stats: Stats | None = None) -> dict:
    ok = [r for r in results if r.status == "ok"]
    lat = [r.latency_s for r in ok]
    span = (max(r.finished_s for r in ok) - min(r.arrival_s for r in ok)) if ok else math.nan
    n_vis = sum(r.n_vis for r in ok)
    out = {"requests": len(results), "served": len(ok), "rejected": len(results) - len(ok),
           "p50_latency_s": percentile(lat, 50), "p99_latency_s": percentile(lat, 99),
           "mean_latency_s": sum(lat) / len(lat) if lat else math.nan,
           "p50_queue_s": percentile([r.admitted_s - r.arrival_s for r in ok], 50),
           "visibilities": n_vis, "span_s": span, "vis_per_s": n_vis / span if span and span > 0 else math.nan}
    if stats is not None:
        out.update({"ticks": stats.ticks, "pieces": stats.pieces, "max_live": stats.max_live,
                    "peak_reserved_bytes": stats.peak_reserved, "gpu_busy_s": stats.gpu_s,
                    "mean_pieces_per_tick": stats.pieces / stats.ticks if stats.ticks else 0.0})
    return out


class GpuExecutor:
    """Runs ticks as fv batches on one stream (torch for buffers and events)."""

    def __init__(self, device: int = 0, n_lanes: int = 8, stream=None):
        import torch
        from . import fv
        self.torch, self.fv = torch, fv
        self.dev = torch.device("cuda", device)
        self.stream = stream or torch.cuda.Stream(device=self.dev)
        # one batch serves every tick: its items are rebuilt per tick, and a tick enqueued while the
        # previous one runs is ordered after it on the stream, so the lane workspaces are never shared
        self.batch = fv.Batch(device=device, stream=self.stream.cuda_stream, n_lanes=n_lanes)

    def elem_bytes(self, plan) -> int:
        return 16 if plan.precision == self.fv.FV_FP64 else 8

    def alloc(self, plan, r: Request):
        nf, nt = r.f_range[1] - r.f_range[0], r.t_range[1] - r.t_range[0]
        dt = self.torch.complex128 if plan.precision == self.fv.FV_FP64 else self.torch.complex64
        return self.torch.empty((nf, nt, plan.n_bl, plan.n_pol), dtype=dt, device=self.dev)

    def free(self, buf) -> None:
        pass                      # released when the caller drops its reference

    def submit(self, work):
        """work: [(plan, out, request, (t, f_lo, f_hi))]; returns a token for wait()."""
        b = self.batch
        b.clear()
        for plan, out, r, (t, f0, f1) in work:
            b.add(plan, out, t_range=(t, t + 1), f_range=(f0, f1),
                  window=(r.f_range[0], r.t_range[0], r.t_range[1] - r.t_range[0]))
        e0 = self.torch.cuda.Event(enable_timing=True)
        e1 = self.torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        b.execute(use_graph=False)
        e1.record(self.stream)
        return (e0, e1)

    def wait(self, token) -> float:
        e0, e1 = token
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3

    def close(self):
        self.batch.close()
