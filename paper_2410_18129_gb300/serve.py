"""Continuous-batching serving loop for constant-time modular exponentiation requests.

A resident pool of moduli of mixed sizes keeps, per size, one Montgomery context and
the window table of each modulus's fixed base on the device (modexp_table_build), so a
fixed-base request (pool entry, exponent) costs only the window loop of Alg. 7; a
variable-base request (pool entry, base, exponent) builds its own table. Requests arrive
over time; the loop

  * admits a batch only while the device bytes of the batches in flight fit a budget
    derived from the free device memory (AdmissionController, re-read as the run goes);
  * keeps one queue per size class and a few batches of each class in flight, and forms the
    next batch of a class from whatever is queued the moment one of its slots frees up
    (continuous batching), so requests that arrive while others run join the very next
    launch of their class, the work of consecutive batches overlaps on the GPU, and a short
    class never waits behind a long one;
  * runs each batch on its slot's stream (one call of the library's mixed entry point: the
    class's fixed-base and variable-base requests), with its result copy and an event;
  * drops requests that waited in the queue longer than a timeout (if one is given);
  * records per-request latency (arrival -> result on the host).

The comparison path (`PlainExecutor`, one slot) serves the same trace one batch at a
time with one launch per size and a synchronisation per batch.
The executor and the clock are parameters, so the loop's host logic is tested on CPU.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

IL = 1


# ------------------------------------------------------------------ host-side logic (no GPU)

class AdmissionController:
    """Byte budget for the batches in flight: min(limit, (free + in flight) * fraction - reserve),
    where free is the free device memory reported by free_fn (injectable). The budget is read
    at start-up and again whenever `refresh` seconds of `clock` have passed since the last
    read (refresh None: read once)."""

    def __init__(self, free_fn=None, fraction: float = 0.5, reserve: int = 1 << 30, limit: int | None = None,
                 refresh: float | None = None, clock=time.perf_counter):
        self.free_fn, self.fraction, self.reserve, self.limit = free_fn, fraction, reserve, limit
        self.refresh, self.clock = refresh, clock
        self.in_use = 0
        self.refused = 0
        self.reads = 0
        self._read()

    def _read(self):
        free = self.free_fn() if self.free_fn is not None else (self.limit or 0)
        budget = int((free + self.in_use) * self.fraction) - self.reserve
        if self.limit is not None:
            budget = min(budget, self.limit) if budget > 0 else self.limit
        self.budget = max(budget, 0)
        self.read_at = self.clock()
        self.reads += 1

    def admit(self, nbytes: int) -> bool:
        if self.refresh is not None and self.clock() - self.read_at >= self.refresh:
            self._read()
        if self.in_use + nbytes > self.budget:
            self.refused += 1
            return False
        self.in_use += nbytes
        return True

    def release(self, nbytes: int):
        self.in_use -= nbytes
        assert self.in_use >= 0


@dataclass(eq=False)
class Handle:
    reqs: np.ndarray
    nbytes: int
    token: object = None
    lane: int = 0        # serve()'s lane index of the batch


@dataclass
class ServeResult:
    latency: np.ndarray          # seconds per request (NaN: timed out in the queue)
    done_at: np.ndarray          # seconds since start (NaN: timed out)
    batches: int
    max_batch_seen: int
    refused: int
    timed_out: int = 0
    results: dict = field(default_factory=dict)

    def summary(self):
        ok = np.isfinite(self.latency)
        lat = self.latency[ok]
        span = float(np.nanmax(self.done_at)) if ok.any() else 0.0
        out = {"requests": int(self.latency.size), "served": int(lat.size), "timed_out": self.timed_out,
               "throughput_per_s": lat.size / span if span > 0 else 0.0, "batches": self.batches,
               "max_batch": self.max_batch_seen, "admission_refusals": self.refused}
        if lat.size:
            out.update({"p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                        "mean_ms": 1e3 * float(lat.mean())})
        return out


def serve(trace, executor, slots: int = 4, max_batch: int = 8192, admission: AdmissionController | None = None,
          clock=time.perf_counter, idle=lambda: None, timeout: float | None = None) -> ServeResult:
    """Replay `trace` (arrival seconds, entries, exponents) in real time through `executor`.
    At most `slots` batches are in flight; a new batch takes the queued requests in arrival
    order, up to max_batch and to what the admission controller allows. Requests still
    queued `timeout` seconds after their arrival are dropped. An executor with a
    completed(handle) method reports the requests of a batch as their results land (each
    call returns those done since the previous one); otherwise a batch completes at once.
    An executor with `lanes` and lane_of(requests) (the continuous executor: one lane per
    size class) gets one queue per lane and `slots` batches in flight per lane: a batch holds
    one lane's requests, so a class waits only for its own batches; the lane whose oldest
    request arrived first is served first."""
    count = len(trace.arrival)
    done_at = np.full(count, np.nan)
    lanes = list(getattr(executor, "lanes", None) or [None])
    lane_of = (executor.lane_of(np.arange(count)) if lanes[0] is not None
               else np.zeros(count, dtype=np.int64))
    key = {ln: i for i, ln in enumerate(lanes)}
    lane_idx = np.array([key[x] for x in lane_of.tolist()], dtype=np.int64) if lanes[0] is not None else lane_of
    queues = [collections.deque() for _ in lanes]
    busy = [0] * len(lanes)
    inflight: list[Handle] = []
    nxt = 0
    completed = 0
    timed_out = 0
    batches = 0
    max_seen = 0
    partial = hasattr(executor, "completed")
    t0 = clock()
    while completed + timed_out < count:
        progressed = False
        now = clock() - t0
        while nxt < count and trace.arrival[nxt] <= now:
            queues[lane_idx[nxt]].append(nxt)
            nxt += 1
        if timeout is not None:
            for queue in queues:
                while queue and now - trace.arrival[queue[0]] > timeout:   # FIFO: the oldest first
                    queue.popleft()
                    timed_out += 1
                    progressed = True
        for h in list(inflight):
            if partial:
                for part in executor.completed(h):
                    done_at[part] = clock() - t0
                    progressed = True
            if executor.done(h):
                if not partial:
                    done_at[h.reqs] = clock() - t0
                completed += h.reqs.size
                if admission is not None:
                    admission.release(h.nbytes)
                executor.finish(h)
                inflight.remove(h)
                busy[h.lane] -= 1
                progressed = True
        order = sorted((trace.arrival[q[0]], i) for i, q in enumerate(queues) if q)
        for _, li in order:
            queue = queues[li]
            while queue and busy[li] < slots:
                take = min(len(queue), max_batch)
                reqs = np.fromiter((queue[i] for i in range(take)), dtype=np.int64, count=take)
                nbytes = executor.bytes_for(reqs)
                if admission is not None:
                    while reqs.size and not admission.admit(nbytes):
                        reqs = reqs[: reqs.size // 2]
                        nbytes = executor.bytes_for(reqs) if reqs.size else 0
                    if not reqs.size:
                        if not inflight:
                            raise RuntimeError("one request needs more device memory than the admission budget")
                        break
                for _ in range(reqs.size):
                    queue.popleft()
                h = executor.submit(reqs, nbytes) if lanes[0] is None else executor.submit(reqs, nbytes, lanes[li])
                h.lane = li
                inflight.append(h)
                busy[li] += 1
                batches += 1
                max_seen = max(max_seen, int(reqs.size))
                progressed = True
        if not progressed:
            if nxt >= count and not inflight and not any(queues):
                break
            idle()
    return ServeResult(done_at - trace.arrival, done_at, batches, max_seen,
                       admission.refused if admission is not None else 0, timed_out,
                       getattr(executor, "results", {}))


# ------------------------------------------------------------------ GPU side

class Pool:
    """Resident moduli with fixed bases: per size a context and its window tables.

    sizes[k] is the bit size of pool entry k; moduli[bits] and bases[bits] hold, in entry
    order, the moduli and fixed bases of the entries of that size (uint32 words, one row
    per entry, bases below their moduli)."""

    def __init__(self, mp, sizes, moduli: dict, bases: dict, windows: dict | None = None):
        import torch
        self.mp, self.torch = mp, torch
        self.sizes = np.asarray(sizes)
        count = self.sizes.size
        self.local = np.zeros(count, dtype=np.int64)
        self.classes = {}
        windows = windows or {}
        dev = lambda x: mp.to_device(mp.interleave(x))
        for bits in sorted(set(int(b) for b in self.sizes)):
            ids = np.nonzero(self.sizes == bits)[0]
            self.local[ids] = np.arange(ids.size)
            N, g = np.asarray(moduli[bits], dtype=np.uint32), np.asarray(bases[bits], dtype=np.uint32)
            if N.shape[0] != ids.size or g.shape != N.shape:
                raise ValueError(f"{bits}-bit entries: {ids.size} in sizes, moduli {N.shape}, bases {g.shape}")
            ctx = mp.MontCtx(dev(N), ids.size, bits, IL)
            w = int(windows.get(bits) or mp.tune_get(bits)["window"])
            tables = torch.empty(mp.modexp_table_bytes(ctx, w) // 4, dtype=torch.int32, device="cuda")
            mp.modexp_table_build(tables, dev(g), ctx, w)
            self.classes[bits] = {"ctx": ctx, "tables": tables, "window": w, "N": N, "g": g, "n": N.shape[1],
                                  "np": mp.modexp_table_bytes(ctx, w) // ((1 << w) * 4 * ids.size), "ids": ids}
        torch.cuda.synchronize()

    def device_bytes(self) -> int:
        return sum(c["tables"].numel() * 4 for c in self.classes.values())

    def request_bytes(self, bits: int, variable: bool = False) -> int:
        c = self.classes[bits]
        words = ((c["n"] + 3) // 4) * 4
        nbytes = 4 * (2 * words + 1)                      # exponent + result (interleaved) + index
        if variable:                                      # its base and its own window table
            nbytes += 4 * words + (1 << c["window"]) * c["np"] * 4
        return nbytes

    def free(self):
        for c in self.classes.values():
            c["ctx"].free()


class _GpuExecutorBase:
    def __init__(self, pool: Pool, trace, keep_results: bool = False):
        self.pool, self.trace, self.mp, self.torch = pool, trace, pool.mp, pool.torch
        self.keep = keep_results
        self.results = {}
        self.bits_of = pool.sizes[trace.entry]
        self.local_of = pool.local[trace.entry]
        bases = getattr(trace, "bases", None)
        self.var = (np.array([b is not None for b in bases], dtype=bool) if bases is not None
                    else np.zeros(len(trace.arrival), dtype=bool))

    def bytes_for(self, reqs) -> int:
        return int(sum(self.pool.request_bytes(int(b), bool(v)) for b, v in zip(self.bits_of[reqs], self.var[reqs])))

    def _class_jobs(self, sel, bits, keep, host_out):
        """Jobs of one size class (its fixed-base and its variable-base requests), with their
        inputs copied to the device on the current stream and result copies queued after."""
        mp, torch = self.mp, self.torch
        c = self.pool.classes[bits]
        jobs, outs = [], []
        for part in (sel[~self.var[sel]], sel[self.var[sel]]):
            if not part.size:
                continue
            variable = bool(self.var[part[0]])
            idx = torch.from_numpy(self.local_of[part].astype(np.uint32).view(np.int32)).pin_memory()
            e = np.stack([self.trace.exponents[i] for i in part])
            ex = torch.from_numpy(mp.interleave(e).view(np.int32)).pin_memory()
            d_idx = idx.to("cuda", non_blocking=True)
            d_ex = ex.to("cuda", non_blocking=True)
            d_y = torch.empty(mp.array_words(IL, part.size, c["n"]), dtype=torch.int32, device="cuda")
            d_base = None
            keep += [idx, ex, d_idx, d_ex, d_y]
            if variable:
                bw = np.stack([self.trace.bases[i] for i in part])
                hb = torch.from_numpy(mp.interleave(bw).view(np.int32)).pin_memory()
                d_base = hb.to("cuda", non_blocking=True)
                keep += [hb, d_base]
            jobs.append((d_y, d_base, d_ex, bits, c["ctx"], c["window"], d_idx, None if variable else c["tables"],
                         part.size))
            outs.append((part, d_y))
        return jobs, outs

    def _copy_back(self, bits, outs, host_out, keep):
        for part, d_y in outs:
            hy = self.torch.empty(d_y.numel(), dtype=self.torch.int32).pin_memory()
            hy.copy_(d_y, non_blocking=True)
            host_out.append((bits, part, hy))
            keep.append(hy)

    def _collect(self, host_out):
        if not self.keep:
            return
        for bits, sel, hy in host_out:
            n = self.pool.classes[bits]["n"]
            words = self.mp.deinterleave(hy.numpy().view(np.uint32), sel.size, n)
            for i, r in enumerate(sel):
                self.results[int(r)] = words[i].copy()


class ContinuousExecutor(_GpuExecutorBase):
    """One lane per size class (serve() keeps a queue and `slots` batches in flight per lane);
    a batch takes one of its class's slots and runs on that slot's stream: async input copies,
    one call of the mixed entry point (the class's fixed-base and variable-base requests),
    async result copies and an event. per_class=False: one set of `slots` slots shared by all
    classes, a batch holding every class (each on its slot's stream for the class); completed()
    then reports a class's requests as soon as its event has fired."""

    def __init__(self, pool, trace, slots: int = 2, keep_results: bool = False, per_class: bool = True):
        super().__init__(pool, trace, keep_results)
        torch = self.torch
        self.streams = {(s, b): torch.cuda.Stream() for s in range(slots) for b in pool.classes}
        if per_class:
            self.lanes = list(pool.classes)
            self.free_slots = {b: list(range(slots)) for b in pool.classes}
        else:
            self.lanes = None
            self.free_slots = {None: list(range(slots))}

    def lane_of(self, reqs):
        return self.bits_of[reqs]

    def submit(self, reqs, nbytes, lane=None):
        torch, mp = self.torch, self.mp
        slot = self.free_slots[lane].pop()
        parts = []
        for bits in self.pool.classes:
            sel = reqs[self.bits_of[reqs] == bits]
            if not sel.size:
                continue
            st = self.streams[(slot, bits)]
            keep, host_out = [], []
            with torch.cuda.stream(st):
                jobs, outs = self._class_jobs(sel, bits, keep, host_out)
                ws = mp.mixed_workspace(jobs)
                keep.append(ws)
                mp.modexp_consttime_mixed(jobs, mp.RED_TRUNCATED, ws)
                self._copy_back(bits, outs, host_out, keep)
                ev = torch.cuda.Event()
                ev.record(st)
            parts.append({"event": ev, "reqs": np.concatenate([p for p, _ in outs]), "keep": keep,
                          "host_out": host_out, "done": False})
        return Handle(reqs, nbytes, {"slot": slot, "lane": lane, "parts": parts})

    def completed(self, h):
        out = []
        for p in h.token["parts"]:
            if not p["done"] and p["event"].query():
                p["done"] = True
                self._collect(p["host_out"])
                p["keep"] = None
                out.append(p["reqs"])
        return out

    def done(self, h) -> bool:
        return all(p["done"] for p in h.token["parts"])

    def finish(self, h):
        self.free_slots[h.token["lane"]].append(h.token["slot"])


class PlainExecutor(_GpuExecutorBase):
    """Comparison path: one launch per size (fixed-base requests with modexp_fixed_base,
    variable-base ones with a one-job mixed call) and a synchronisation per batch."""

    def submit(self, reqs, nbytes):
        torch, mp = self.torch, self.mp
        host_out, keep = [], []
        for bits in self.pool.classes:
            sel = reqs[self.bits_of[reqs] == bits]
            if not sel.size:
                continue
            c = self.pool.classes[bits]
            jobs, outs = self._class_jobs(sel, bits, keep, host_out)
            for job in jobs:
                d_y, d_base, d_ex, _, ctx, w, d_idx, tables, nreq = job
                if tables is not None:
                    mp.modexp_fixed_base(d_y, d_idx, d_ex, bits, nreq, ctx, tables, w)
                else:
                    mp.modexp_consttime_mixed([job], mp.RED_TRUNCATED, mp.mixed_workspace([job]))
            self._copy_back(bits, outs, host_out, keep)
        torch.cuda.synchronize()
        self._collect(host_out)
        return Handle(reqs, nbytes, {})

    def done(self, h) -> bool:
        return True

    def finish(self, h):
        pass
