"""Serving loop host logic on CPU: admission by memory budget, continuous batching, slot
limits and latency accounting, with a fake executor and a fake clock (no GPU)."""
import importlib.util
import os
import sys

import numpy as np

import seeded_inputs as si

# serve.py's host logic needs only numpy; load it by path so that this CPU test does not
# need the built CUDA library (the package refuses to import without it)
_spec = importlib.util.spec_from_file_location(
    "mpgpu_serve", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                "paper_2410_18129_gb300", "serve.py"))
_serve = importlib.util.module_from_spec(_spec)
sys.modules["mpgpu_serve"] = _serve          # dataclasses look their module up here
_spec.loader.exec_module(_serve)
AdmissionController, Handle, serve = _serve.AdmissionController, _serve.Handle, _serve.serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def advance(self, dt=1e-4):
        self.t += dt


class FakeExecutor:
    """Each batch takes `base + per_req * size` seconds of fake time; records what it saw."""

    def __init__(self, clock, base=0.01, per_req=1e-5, req_bytes=100, budget_check=None):
        self.clock, self.base, self.per_req, self.req_bytes = clock, base, per_req, req_bytes
        self.inflight = 0
        self.max_inflight = 0
        self.bytes_now = 0
        self.max_bytes = 0
        self.batches = []
        self.results = {}

    def bytes_for(self, reqs):
        return int(reqs.size * self.req_bytes)

    def submit(self, reqs, nbytes):
        self.inflight += 1
        self.max_inflight = max(self.max_inflight, self.inflight)
        self.bytes_now += nbytes
        self.max_bytes = max(self.max_bytes, self.bytes_now)
        self.batches.append((self.clock(), reqs.copy()))
        return Handle(reqs, nbytes, {"end": self.clock() + self.base + self.per_req * reqs.size})

    def done(self, h):
        return self.clock() >= h.token["end"]

    def finish(self, h):
        self.inflight -= 1
        self.bytes_now -= h.nbytes


def trace(rate, count, seed=0):
    sizes = np.full(16, 1024)
    return si.poisson_trace(seed, rate, count, sizes)


def test_admission_budget_from_free_memory():
    a = AdmissionController(free_fn=lambda: 10_000, fraction=0.5, reserve=1000)
    assert a.budget == 4000
    assert a.admit(3000) and not a.admit(1500) and a.refused == 1
    a.release(3000)
    assert a.admit(4000)
    b = AdmissionController(free_fn=lambda: 10 ** 12, fraction=0.5, reserve=0, limit=777)
    assert b.budget == 777


def test_every_request_completes_with_consistent_latency():
    clk = FakeClock()
    ex = FakeExecutor(clk)
    tr = trace(2e4, 3000)
    res = serve(tr, ex, slots=3, max_batch=256, clock=clk, idle=clk.advance)
    assert np.isfinite(res.latency).all() and (res.latency > 0).all()
    assert np.allclose(res.done_at - tr.arrival, res.latency)
    served = np.sort(np.concatenate([b for _, b in ex.batches]))
    assert (served == np.arange(3000)).all()                 # each request exactly once
    assert ex.max_inflight <= 3
    assert max(b.size for _, b in ex.batches) <= 256


def test_continuous_batching_admits_arrivals_while_busy():
    """Requests that arrive while batches run are taken as soon as a slot frees, in arrival
    order; with one slot the next batch starts right when the previous one ends."""
    clk = FakeClock()
    ex = FakeExecutor(clk, base=0.05, per_req=0.0)
    tr = trace(1e4, 2000)
    serve(tr, ex, slots=1, max_batch=10 ** 6, clock=clk, idle=clk.advance)
    starts = [t for t, _ in ex.batches]
    sizes = [b.size for _, b in ex.batches]
    assert sizes[0] < sizes[1]                 # the first batch is small, later ones carry the queue
    assert all(abs((s2 - s1) - 0.05) < 2e-3 for s1, s2 in zip(starts[1:-1], starts[2:]))
    order = np.concatenate([b for _, b in ex.batches])
    assert (order == np.arange(2000)).all()    # FIFO


def test_admission_limits_bytes_in_flight():
    clk = FakeClock()
    ex = FakeExecutor(clk, req_bytes=1000)
    adm = AdmissionController(limit=50_000, reserve=0, fraction=1.0)
    tr = trace(1e5, 4000)
    res = serve(tr, ex, slots=8, max_batch=1000, admission=adm, clock=clk, idle=clk.advance)
    assert ex.max_bytes <= 50_000
    assert res.refused > 0 and adm.in_use == 0


def test_poisson_trace_statistics():
    sizes = si.pool_sizes(0, 4096)
    assert {b: int((sizes == b).sum()) for b in (1024, 2048, 3072, 4096)} == \
        {1024: 1024, 2048: 1639, 3072: 819, 4096: 614}
    tr = si.poisson_trace(0, 5e4, 20000, sizes)
    gaps = np.diff(tr.arrival)
    assert abs(gaps.mean() * 5e4 - 1) < 0.03
    assert (gaps >= 0).all()
    counts = np.bincount(tr.entry, minlength=4096)
    assert counts.max() < 20 and (tr.entry < 4096).all()
    assert all(e.shape[0] == (int(sizes[k]) + 31) // 32 for e, k in zip(tr.exponents[:50], tr.entry[:50]))


class PartialExecutor(FakeExecutor):
    """Like FakeExecutor, but the requests of a batch land in two parts: the first half after
    `base`, the rest after `base + late` (a slow size class)."""

    def __init__(self, clock, base=0.01, late=0.05):
        super().__init__(clock, base=base, per_req=0.0)
        self.late = late

    def submit(self, reqs, nbytes):
        h = super().submit(reqs, nbytes)
        t = self.clock()
        half = reqs.size // 2
        h.token = {"parts": [[reqs[:half], t + self.base, False], [reqs[half:], t + self.base + self.late, False]]}
        return h

    def completed(self, h):
        out = []
        for p in h.token["parts"]:
            if not p[2] and self.clock() >= p[1]:
                p[2] = True
                out.append(p[0])
        return out

    def done(self, h):
        return all(p[2] for p in h.token["parts"])


def test_requests_complete_with_their_part_of_a_batch():
    """A request's latency ends when its own part of the batch lands, not the whole batch."""
    clk = FakeClock()
    ex = PartialExecutor(clk, base=0.01, late=0.05)
    tr = trace(2e3, 400)
    res = serve(tr, ex, slots=2, max_batch=64, clock=clk, idle=clk.advance)
    assert np.isfinite(res.latency).all()
    early, late = [], []
    for start, b in ex.batches:
        half = b.size // 2
        early += list(res.done_at[b[:half]] - start)
        late += list(res.done_at[b[half:]] - start)
    assert max(early) < 0.02 and min(late) > 0.055


def test_queued_requests_time_out():
    """With one slot and slow batches the queue grows; requests older than the timeout are
    dropped before they are batched (never sent to the executor), the rest are served."""
    clk = FakeClock()
    ex = FakeExecutor(clk, base=0.2, per_req=0.0)
    tr = trace(5e3, 3000)
    res = serve(tr, ex, slots=1, max_batch=100, clock=clk, idle=clk.advance, timeout=0.1)
    sent = np.concatenate([b for _, b in ex.batches])
    assert res.timed_out > 0 and res.timed_out + sent.size == 3000
    assert np.isnan(res.latency).sum() == res.timed_out
    starts = {int(r): t for t, b in ex.batches for r in b}
    assert all(starts[r] - tr.arrival[r] <= 0.1 + 1e-3 for r in sent)
    s = res.summary()
    assert s["served"] == sent.size and s["timed_out"] == res.timed_out


def test_admission_budget_is_read_again():
    """The budget follows the free memory read every `refresh` seconds (fake clock)."""
    clk = FakeClock()
    free = {"v": 10_000}
    a = AdmissionController(free_fn=lambda: free["v"], fraction=0.5, reserve=0, refresh=1.0, clock=clk)
    assert a.budget == 5000 and a.admit(4000)
    free["v"] = 2_000                     # another user took memory: in flight 4000 + free 2000
    assert not a.admit(2000)              # not re-read yet (budget 5000)
    clk.advance(1.0)
    assert not a.admit(1) or a.budget == 3000
    assert a.budget == 3000 and a.reads == 2
    a.release(4000)
    free["v"] = 20_000
    clk.advance(1.0)
    assert a.admit(9000) and a.budget == 10_000


def test_variable_base_trace():
    pool = si.serving_pool(0, 64)
    tr = si.poisson_trace(0, 1e4, 500, pool.sizes)
    tv = si.with_bases(tr, pool, 0.3)
    var = [k for k, b in enumerate(tv.bases) if b is not None]
    assert 100 < len(var) < 200
    for k in var[:40]:
        bits = int(pool.sizes[tv.entry[k]])
        ids = np.nonzero(pool.sizes == bits)[0]
        N = pool.moduli[bits][int(np.nonzero(ids == tv.entry[k])[0][0])]
        b = tv.bases[k]
        assert b.shape == N.shape and int("".join(f"{w:08x}" for w in b[::-1]), 16) < \
            int("".join(f"{w:08x}" for w in N[::-1]), 16)


class LaneExecutor(FakeExecutor):
    """Requests with index divisible by 4 are 'slow' (a batch holding one takes 0.2 s of fake
    time), the others 'fast' (0.01 s). With lanes, serve() keeps one queue per kind."""

    def __init__(self, clock, lanes=True):
        super().__init__(clock)
        self.lanes = ["fast", "slow"] if lanes else None
        self.busy = {"fast": 0, "slow": 0, None: 0}
        self.max_busy = dict(self.busy)

    def lane_of(self, reqs):
        return np.where(np.asarray(reqs) % 4 == 0, "slow", "fast")

    def submit(self, reqs, nbytes, lane=None):
        h = super().submit(reqs, nbytes)
        slow = bool((reqs % 4 == 0).any())
        h.token = {"end": self.clock() + (0.2 if slow else 0.01), "lane": lane}
        self.busy[lane] += 1
        self.max_busy[lane] = max(self.max_busy[lane], self.busy[lane])
        return h

    def finish(self, h):
        super().finish(h)
        self.busy[h.token["lane"]] -= 1


def test_lanes_keep_a_fast_class_off_a_slow_one():
    """With one lane per class a batch holds one class and each class has its own slots, so
    the fast class is served within its own batch time while slow batches are in flight;
    without lanes the same requests wait behind batches that hold a slow request."""
    tr = trace(2e3, 400, seed=3)
    fast = np.arange(400) % 4 != 0
    clk = FakeClock()
    ex = LaneExecutor(clk)
    res = serve(tr, ex, slots=2, max_batch=64, clock=clk, idle=clk.advance)
    assert np.isfinite(res.latency).all()
    for _, b in ex.batches:
        assert len(set(ex.lane_of(b).tolist())) == 1               # one class per batch
    assert ex.max_busy["fast"] <= 2 and ex.max_busy["slow"] <= 2 and ex.max_busy["slow"] >= 1
    assert np.percentile(res.latency[fast], 90) < 0.05
    clk2 = FakeClock()
    ex2 = LaneExecutor(clk2, lanes=False)
    res2 = serve(tr, ex2, slots=2, max_batch=64, clock=clk2, idle=clk2.advance)
    assert np.isfinite(res2.latency).all()
    assert np.percentile(res2.latency[fast], 90) > 0.1
