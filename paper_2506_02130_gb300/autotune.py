"""Autotuner for batched slices: route, upsampling factor, spreading form, FFT radix and bin shape.

The paper exposes only the tolerance eps; the grid sizes follow from it
(Eq. 5) once the upsampling factor sigma and the kernel width w are fixed
(Section 2.2).  A smaller sigma shrinks the FFT (length sigma * nf1 per
dimension) but widens the kernel (w grows as 1/sqrt(1 - 1/sigma) for the same
eps), so spreading and interpolation cost more: which wins depends on the
ratio of sources and targets to grid cells, i.e. on the array, the sky and the
frequency.  The tuner times each candidate on a representative slice of every
class of slices and keeps the fastest.

Candidates (each meets the slice's transform tolerance by its choice of w):
  * sigma: 1.25 or 2 on the FP64 path; 1.5 or 2 on the mixed path, because the
    two deconvolutions amplify FP32 rounding too much at 1.25 (the plan
    rejects mixed plans below 1.5);
  * spreading tile: "gather" (the tile's sorted sources staged in shared
    memory; on the mixed path's two-dimensional grids a persistent ring of
    32 x 16-cell tiles, one warp per 8 x 8 block) or "scatter" (32 x 16-cell
    tiles, one warp per source, shared-memory atomics).  The tensor-core form
    of the gather is an explicit option, not a candidate;
  * FFT radix cap: 8 or 16 (the largest butterfly held in registers);
  * route (when the tuner is asked to choose it): "auto" (the lattice route of
    Section 2.2.1 when the array is a lattice and its grid is the smaller,
    else type-3) or "type3".  By default only "auto": a slice timed alone is
    not a batch, and measured on the 2,048-slice batch (8 lanes) the slices
    that timed faster alone on type-3 made the batch 18% slower than on the
    lattice route, whose smaller kernels overlap better;
  * bin shape of the per-time source sort (cells of the highest channel's grid
    per bin): 8 x 4, 4 x 4, 8 x 8 or 16 x 4, tried in a second round for the
    winner when it is a type-3 plan with a gather spreading (the bins decide
    how many candidate sources each spreading tile stages).

Classes group slices by precision, antenna count and source-count octave, so
one measurement covers every slice of similar cost.  The choices are kept in
a dictionary that can be saved to and loaded from JSON.
"""
from __future__ import annotations

import json
import math
from dataclasses import asdict, dataclass
from typing import Callable, Iterable

from . import fv


@dataclass(frozen=True)
class Choice:
    upsampfac: float
    spread: str
    fft_max_radix: int
    transform: str = "auto"
    bin_size: tuple = (0, 0)

    def plan_kwargs(self) -> dict:
        return {"upsampfac": self.upsampfac, "spread": self.spread, "fft_max_radix": self.fft_max_radix,
                "transform": self.transform, "bin_size": tuple(self.bin_size)}


DEFAULT = {fv.FV_FP64: Choice(2.0, "gather", 16), fv.FV_MIXED: Choice(2.0, "gather", 16)}

BIN_SHAPES = ((4, 4), (8, 8), (16, 4))


def candidates(precision: int, routes=("auto",)) -> list[Choice]:
    sig = (1.25, 2.0) if precision == fv.FV_FP64 else (1.5, 2.0)
    return [Choice(s, sp, r, tr) for tr in routes for s in sig for sp in ("gather", "scatter") for r in (8, 16)]


def bin_candidates(best: Choice) -> list[Choice]:
    """Second round: other bin shapes for a type-3 plan with the gather spreading."""
    if best.spread != "gather":
        return []
    return [Choice(best.upsampfac, best.spread, best.fft_max_radix, "type3", b) for b in BIN_SHAPES]


def class_key(precision: int, n_ant: int, n_src: int) -> str:
    """Slices of one precision and array whose source counts share an octave."""
    octave = int(math.floor(math.log2(max(n_src, 1))))
    return f"{'fp64' if precision == fv.FV_FP64 else 'mixed'}/ant{n_ant}/src2^{octave}"


class Autotuner:
    """Picks a Choice per class by timing; `timer(choice, slice)` returns the seconds, or (seconds, route)
    with the route the plan took ("type3", "lattice", ...)."""

    def __init__(self, timer: Callable | None = None, routes=("auto",)):
        self.table: dict[str, Choice] = {}
        self.timings: dict[str, dict[str, float]] = {}
        self.timer = timer
        self.routes = tuple(routes)

    def choice(self, precision: int, n_ant: int, n_src: int) -> Choice:
        return self.table.get(class_key(precision, n_ant, n_src), DEFAULT[precision])

    def tune(self, slices: Iterable, key_of: Callable, precision_of: Callable) -> dict[str, Choice]:
        """Time every candidate on one representative slice per untuned class
        (the member with the median source count)."""
        groups: dict[str, list] = {}
        for s in slices:
            groups.setdefault(key_of(s), []).append(s)
        for key, members in groups.items():
            if key in self.table:
                continue
            members = sorted(members, key=lambda s: s.problem.sky.n_src)
            rep = members[len(members) // 2]
            times, routes = {}, {}

            def measure(c):
                try:
                    r = self.timer(c, rep)
                except fv.FvError:
                    return            # a candidate the plan rejects (grid or FFT too large) is skipped
                times[c], routes[c] = (r[0], r[1]) if isinstance(r, tuple) else (r, c.transform)

            for c in candidates(precision_of(rep), self.routes):
                measure(c)
            if not times:
                continue
            best = min(times, key=times.get)
            # "auto" resolves to the lattice route or type-3; only a type-3 winner has bins to tune
            if routes[best] == "type3":
                for c in bin_candidates(best):
                    measure(c)
                best = min(times, key=times.get)
            self.table[key] = best
            self.timings[key] = {json.dumps(asdict(c)): t for c, t in times.items()}
        return self.table

    def save(self, path: str) -> None:
        with open(path, "w") as f:
            json.dump({k: asdict(v) for k, v in self.table.items()}, f, indent=1, sort_keys=True)

    def load(self, path: str) -> None:
        with open(path) as f:
            self.table.update({k: Choice(**{**v, "bin_size": tuple(v.get("bin_size", (0, 0)))})
                               for k, v in json.load(f).items()})


def precision_of(bs) -> int:
    return fv.FV_FP64 if bs.precision == "fp64" else fv.FV_MIXED


def key_of(bs) -> str:
    return class_key(precision_of(bs), len(bs.problem.ant_enu), bs.problem.sky.n_src)


def cuda_timer(stream, reps: int = 3, warmup: int = 1):
    """A timer that builds a plan for the choice, runs the slice `warmup` times,
    then returns the mean device time of `reps` runs (CUDA events on `stream`)."""
    import torch

    def timer(choice: Choice, bs) -> float:
        prob = bs.problem
        prec = precision_of(bs)
        p = fv.Plan.from_problem(prob, precision=prec, eps=bs.nufft_eps, stream=stream.cuda_stream, n_streams=1,
                                 **choice.plan_kwargs())
        try:
            p.set_sky(prob.sky.ra, prob.sky.dec, prob.sky.flux)
            out = torch.empty(p.out_shape, dtype=torch.complex128 if prec == fv.FV_FP64 else torch.complex64,
                              device=torch.device("cuda", torch.cuda.current_device()))
            for _ in range(warmup):
                p.run(out)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                p.run(out)
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / 1e3 / reps, p.info()["transform"]
        finally:
            p.close()

    return timer
