"""Continuous-batching serving loop for constant-time modular exponentiation requests.

A resident pool of moduli of mixed sizes keeps, per size, one Montgomery context and
the window table of each modulus's fixed base on the device (modexp_table_build), so a
request (pool entry, exponent) costs only the window loop of Alg. 7. Requests arrive
over time; the loop

  * admits a batch only while the device bytes of the batches in flight fit a budget
    derived from the free device memory at start-up (AdmissionController);
  * keeps several batches in flight on separate CUDA streams and forms the next batch
    from whatever is queued the moment a stream slot frees up (continuous batching), so
    requests that arrive while others run join the very next launch and the work of
    consecutive batches overlaps on the GPU;
  * runs every batch, whatever its size mix, as one persistent launch with fixed-base jobs
    (modexp_consttime_mixed), with its host<->device copies on the same stream;
  * records per-request latency (arrival -> result on the host).

The comparison path (`PlainExecutor`, one slot) serves the same trace one batch at a
time with one launch per size (modexp_fixed_base) and a synchronisation per batch.
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
    """Byte budget for the batches in flight: min(limit, free * fraction - reserve), with the
    free device memory read once at start-up (free_fn is injectable)."""

    def __init__(self, free_fn=None, fraction: float = 0.5, reserve: int = 1 << 30, limit: int | None = None):
        free = free_fn() if free_fn is not None else (limit or 0)
        budget = int(free * fraction) - reserve
        if limit is not None:
            budget = min(budget, limit) if budget > 0 else limit
        self.budget = max(budget, 0)
        self.in_use = 0
        self.refused = 0

    def admit(self, nbytes: int) -> bool:
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


@dataclass
class ServeResult:
    latency: np.ndarray          # seconds per request
    done_at: np.ndarray          # seconds since start
    batches: int
    max_batch_seen: int
    refused: int
    results: dict = field(default_factory=dict)

    def summary(self):
        lat = self.latency
        span = float(self.done_at.max()) if self.done_at.size else 0.0
        return {"requests": int(lat.size), "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mean_ms": 1e3 * float(lat.mean()),
                "throughput_per_s": lat.size / span if span > 0 else 0.0, "batches": self.batches,
                "max_batch": self.max_batch_seen, "admission_refusals": self.refused}


def serve(trace, executor, slots: int = 4, max_batch: int = 8192, admission: AdmissionController | None = None,
          clock=time.perf_counter, idle=lambda: None) -> ServeResult:
    """Replay `trace` (arrival seconds, entries, exponents) in real time through `executor`.
    At most `slots` batches are in flight; a new batch takes the queued requests in arrival
    order, up to max_batch and to what the admission controller allows."""
    count = len(trace.arrival)
    done_at = np.full(count, np.nan)
    queue = collections.deque()
    inflight: list[Handle] = []
    nxt = 0
    completed = 0
    batches = 0
    max_seen = 0
    t0 = clock()
    while completed < count:
        progressed = False
        now = clock() - t0
        while nxt < count and trace.arrival[nxt] <= now:
            queue.append(nxt)
            nxt += 1
        for h in list(inflight):
            if executor.done(h):
                t = clock() - t0
                done_at[h.reqs] = t
                completed += h.reqs.size
                if admission is not None:
                    admission.release(h.nbytes)
                executor.finish(h)
                inflight.remove(h)
                progressed = True
        while queue and len(inflight) < slots:
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
            inflight.append(executor.submit(reqs, nbytes))
            batches += 1
            max_seen = max(max_seen, int(reqs.size))
            progressed = True
        if not progressed:
            if nxt >= count and not inflight and not queue:
                break
            idle()
    return ServeResult(done_at - trace.arrival, done_at, batches, max_seen,
                       admission.refused if admission is not None else 0,
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
                                  "ids": ids}
        torch.cuda.synchronize()

    def device_bytes(self) -> int:
        return sum(c["tables"].numel() * 4 for c in self.classes.values())

    def request_bytes(self, bits: int) -> int:
        n = self.classes[bits]["n"]
        return 4 * (2 * ((n + 3) // 4) * 4 + 1)   # exponent + result (interleaved) + index

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

    def bytes_for(self, reqs) -> int:
        return int(sum(self.pool.request_bytes(int(b)) for b in self.bits_of[reqs]))

    def _pack(self, reqs):
        """Per size: (bits, request ids, pinned index, pinned exponents, result words)."""
        mp, torch = self.mp, self.torch
        out = []
        for bits in self.pool.classes:
            sel = reqs[self.bits_of[reqs] == bits]
            if not sel.size:
                continue
            n = self.pool.classes[bits]["n"]
            idx = torch.from_numpy(self.local_of[sel].astype(np.uint32).view(np.int32)).pin_memory()
            e = np.stack([self.trace.exponents[i] for i in sel])
            ex = torch.from_numpy(mp.interleave(e).view(np.int32)).pin_memory()
            out.append((bits, sel, idx, ex, mp.array_words(IL, sel.size, n)))
        return out

    def _collect(self, h):
        if not self.keep:
            return
        for bits, sel, hy in h.token["host_out"]:
            n = self.pool.classes[bits]["n"]
            words = self.mp.deinterleave(hy.numpy().view(np.uint32), sel.size, n)
            for i, r in enumerate(sel):
                self.results[int(r)] = words[i].copy()

    def finish(self, h):
        self._collect(h)


class ContinuousExecutor(_GpuExecutorBase):
    """Each batch: async copies, ONE mixed persistent launch with fixed-base jobs, async
    result copy, all on the batch's own stream; done() polls its event."""

    def __init__(self, pool, trace, slots: int = 4, keep_results: bool = False):
        super().__init__(pool, trace, keep_results)
        self.streams = [self.torch.cuda.Stream() for _ in range(slots)]
        self.free_streams = list(range(slots))

    def submit(self, reqs, nbytes):
        torch, mp = self.torch, self.mp
        si = self.free_streams.pop()
        st = self.streams[si]
        packs = self._pack(reqs)
        keep = []
        host_out = []
        with torch.cuda.stream(st):
            jobs = []
            for bits, sel, idx, ex, words in packs:
                c = self.pool.classes[bits]
                d_idx = idx.to("cuda", non_blocking=True)
                d_ex = ex.to("cuda", non_blocking=True)
                d_y = torch.empty(words, dtype=torch.int32, device="cuda")
                jobs.append((d_y, None, d_ex, bits, c["ctx"], c["window"], d_idx, c["tables"], sel.size))
                keep += [idx, ex, d_idx, d_ex, d_y]
            ws = torch.empty(64, dtype=torch.int32, device="cuda")   # tile counter only
            mp.modexp_consttime_mixed(jobs, mp.RED_TRUNCATED, ws)
            for (bits, sel, *_), job in zip(packs, jobs):
                hy = torch.empty(job[0].numel(), dtype=torch.int32).pin_memory()
                hy.copy_(job[0], non_blocking=True)
                host_out.append((bits, sel, hy))
            ev = torch.cuda.Event()
            ev.record(st)
        keep.append(ws)
        return Handle(reqs, nbytes, {"event": ev, "stream": si, "keep": keep, "host_out": host_out})

    def done(self, h) -> bool:
        return h.token["event"].query()

    def finish(self, h):
        super().finish(h)
        self.free_streams.append(h.token["stream"])
        h.token["keep"] = None


class PlainExecutor(_GpuExecutorBase):
    """Comparison path: one launch per size (modexp_fixed_base) and a synchronisation per batch."""

    def submit(self, reqs, nbytes):
        torch, mp = self.torch, self.mp
        host_out = []
        for bits, sel, idx, ex, words in self._pack(reqs):
            c = self.pool.classes[bits]
            d_y = torch.empty(words, dtype=torch.int32, device="cuda")
            mp.modexp_fixed_base(d_y, idx.cuda(), ex.cuda(), bits, sel.size, c["ctx"], c["tables"], c["window"])
            host_out.append((bits, sel, d_y.cpu()))
        torch.cuda.synchronize()
        return Handle(reqs, nbytes, {"host_out": host_out})

    def done(self, h) -> bool:
        return True
