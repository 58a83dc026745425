"""Host logic of the serving loop with a simulated GPU (no device): every
request's slices are covered exactly once, admission respects the HBM budget
and arrival order, requests that arrive while others run join later ticks,
oversize requests are rejected, and the latency percentiles are right."""
import collections
import random

import numpy as np
import pytest

from paper_2506_02130_gb300 import serve


class FakePlan:
    def __init__(self, n_bl, n_pol=1, n_freq=16, n_time=8, precision=1):
        self.n_bl, self.n_pol, self.n_freq, self.n_time, self.precision = n_bl, n_pol, n_freq, n_time, precision


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeExecutor:
    """Runs a tick instantly on the host; wait() advances the simulated clock by its cost."""

    def __init__(self, clock, slice_s):
        self.clock, self.slice_s = clock, slice_s
        self.cover = collections.defaultdict(list)
        self.ticks = []

    def elem_bytes(self, plan):
        return 8

    def alloc(self, plan, r):
        return {"rid": r.rid}

    def free(self, buf):
        buf["freed"] = True

    def submit(self, work):
        cost = 0.0
        rids = []
        for plan, out, r, (t, f0, f1) in work:
            assert r.t_range[0] <= t < r.t_range[1] and r.f_range[0] <= f0 < f1 <= r.f_range[1]
            for f in range(f0, f1):
                self.cover[r.rid].append((t, f))
            cost += (f1 - f0) * self.slice_s[r.kind]
            rids.append(r.rid)
        self.ticks.append(rids)
        return cost

    def wait(self, cost):
        self.clock.t += cost
        return cost


def _requests(n, rate, seed=0):
    rng = random.Random(seed)
    t, out = 0.0, []
    for i in range(n):
        t += rng.expovariate(rate)
        kind = rng.choice(["small", "big"])
        nf = rng.randint(1, 16)
        f0 = rng.randint(0, 16 - nf)
        nt = rng.randint(1, 8)
        t0 = rng.randint(0, 8 - nt)
        out.append(serve.Request(i, t, kind, (f0, f0 + nf), (t0, t0 + nt)))
    return out


def _server(budget, clock, max_live=64, tick_s=0.01):
    plans = {"small": FakePlan(100), "big": FakePlan(1000, n_pol=4)}
    slice_s = {"small": 1e-4, "big": 1e-3}
    ex = FakeExecutor(clock, slice_s)
    return serve.Server(plans, ex, budget, slice_s, max_live=max_live, tick_s=tick_s), ex


def test_every_slice_once_and_budget_respected():
    clock = Clock()
    srv, ex = _server(budget=6_000_000, clock=clock)     # one full-size "big" request is 4 MB
    reqs = _requests(60, rate=200.0)
    res = srv.run(reqs, clock=clock, sleep=clock.sleep)
    assert len(res) == len(reqs)
    assert all(r.status == "ok" for r in res)
    for r in reqs:
        want = sorted((t, f) for t in range(*r.t_range) for f in range(*r.f_range))
        assert sorted(ex.cover[r.rid]) == want
    assert srv.stats.peak_reserved <= 6_000_000
    for r, q in zip(res, reqs):
        assert r.finished_s >= r.admitted_s >= r.arrival_s - 1e-12
        assert r.n_vis == q.n_slices * srv.plans[q.kind].n_bl * srv.plans[q.kind].n_pol


def test_admission_in_arrival_order_and_slots():
    clock = Clock()
    srv, ex = _server(budget=10 ** 12, clock=clock, max_live=3)
    reqs = _requests(40, rate=2000.0, seed=3)
    res = srv.run(reqs, clock=clock, sleep=clock.sleep)
    adm = [r.admitted_s for r in sorted(res, key=lambda r: r.arrival_s)]
    assert adm == sorted(adm)
    assert srv.stats.max_live <= 3


def test_continuous_batching_mixes_requests_in_ticks():
    clock = Clock()
    srv, ex = _server(budget=10 ** 12, clock=clock, tick_s=0.002)
    # a long request first, short ones arriving while it runs
    reqs = [serve.Request(0, 0.0, "big", (0, 16), (0, 8))]
    reqs += [serve.Request(i, 0.01 * i, "small", (0, 2), (0, 1)) for i in range(1, 6)]
    res = srv.run(reqs, clock=clock, sleep=clock.sleep)
    # the short requests finish before the long one: they did not wait for it to drain
    assert all(r.finished_s < res[0].finished_s for r in res[1:])
    assert any(0 in t and len(t) > 1 for t in ex.ticks)


def test_oversize_request_is_rejected_and_the_rest_served():
    clock = Clock()
    srv, ex = _server(budget=500_000, clock=clock)
    reqs = [serve.Request(0, 0.0, "big", (0, 16), (0, 8)),     # 16*8*1000*4*8 B > budget
            serve.Request(1, 0.0, "small", (0, 4), (0, 2))]
    res = srv.run(reqs, clock=clock, sleep=clock.sleep)
    assert res[0].status.startswith("rejected")
    assert res[1].status == "ok"
    s = serve.summary(res, srv.stats)
    assert s["served"] == 1 and s["rejected"] == 1


def test_budget_blocks_until_memory_frees():
    clock = Clock()
    srv, ex = _server(budget=16 * 8 * 1000 * 4 * 8, clock=clock)   # exactly one big request fits
    reqs = [serve.Request(i, 0.0, "big", (0, 16), (0, 8)) for i in range(3)]
    res = srv.run(reqs, clock=clock, sleep=clock.sleep)
    assert srv.stats.max_live == 1
    assert res[0].finished_s <= res[1].admitted_s + 1e-12
    assert res[1].finished_s <= res[2].admitted_s + 1e-12


@pytest.mark.parametrize("q", [0, 1, 50, 90, 99, 100])
def test_percentile_matches_numpy(q):
    xs = list(np.random.default_rng(1).exponential(1.0, 101))
    assert serve.percentile(xs, q) == pytest.approx(np.percentile(xs, q))
