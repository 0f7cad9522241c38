"""Autotuner: per operand size, pick the group shape (threads per instance G x words per
thread M), the exponentiation window (4..6), the window-table placement (global or shared
memory), whether the Montgomery products of the truncated reduction use the truncated
Karatsuba form, and the schoolbook/Karatsuba choice for products, by timing the library's own kernels on this GPU, each on whole residency rounds of
its own; apply the choice through mp_tune_set / mp_tune_set_table / mp_tune_set_mont_karatsuba
and cache it as
JSON keyed by GPU name, SM count and size.

    import paper_2410_18129_gb300.tune as tune
    choice = tune.load_or_tune(sizes=(1024, 2048, 3072, 4096))   # times, caches, applies

Timing: CUDA events on the current stream after one warm-up launch, full-length
exponents, a probe batch of two whole residency rounds of the kernel being timed.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

import paper_2410_18129_gb300 as mp

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tune_cache.json")
NEVER = 0xFFFFFFFF   # "never use Karatsuba for AUTO products"


def _key():
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|{p.multi_processor_count}"


def _time(fn, reps=1):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _probe(bits: int, batch: int, seed: int = 7):
    """Synthetic probe operands (device, interleaved): odd moduli with the top bit set,
    bases below N, full-length exponents. Values do not change the timing."""
    n = (bits + 31) // 32
    rng = np.random.Generator(np.random.PCG64(seed + bits))
    N = rng.integers(0, 1 << 32, size=(batch, n), dtype=np.uint64).astype(np.uint32)
    top = bits - 32 * (n - 1)
    if top < 32:
        N[:, -1] &= np.uint32((1 << top) - 1)
    N[:, -1] |= np.uint32(1 << (top - 1))
    N[:, 0] |= np.uint32(1)
    a = N.copy()
    a[:, -1] >>= np.uint32(1)                     # a < N
    e = rng.integers(0, 1 << 32, size=(batch, n), dtype=np.uint64).astype(np.uint32)
    if top < 32:
        e[:, -1] &= np.uint32((1 << top) - 1)
    dev = lambda x: mp.to_device(mp.interleave(x))
    return dev(N), dev(a), dev(e)


def tune(sizes=(1024, 2048, 3072, 4096), windows=(4, 5, 6), rounds: int = 2, log=None):
    """Time every (shape, window) for each size, the truncated Karatsuba form of the Montgomery
    products against the best schoolbook choice, and both product algorithms; returns the
    choice per size (not applied). Each kernel is timed on a probe batch of `rounds` whole
    residency rounds of its own (mp_shape_residency x SMs), so that no kernel is measured on a
    partial last round."""
    IL = mp.LAYOUT_INTERLEAVED
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out = {}
    for bits in sizes:
        cands = mp.shape_candidates(bits)
        per_sm = {(G, M): mp.shape_residency(bits, G, M) for G, M in cands}
        try:
            per_sm_tk = mp.shape_residency(bits, algo=mp.ALGO_KARATSUBA)
        except mp.MpError:
            per_sm_tk = 0
        Bmax = rounds * sms * max(list(per_sm.values()) + [per_sm_tk])
        N, A, E = _probe(bits, Bmax)
        ctxs = {}

        def ctx_for(B):
            if B not in ctxs:
                ctxs[B] = mp.MontCtx(N, B, bits, IL) if B == Bmax else mp.MontCtx(
                    mp.to_device(mp.interleave(mp.deinterleave(mp.to_host(N), Bmax, (bits + 31) // 32)[:B])), B, bits, IL)
            return ctxs[B]

        Y = torch.zeros_like(A)
        timings = {}
        best = None
        for G, M in cands:
            B = rounds * sms * per_sm[(G, M)]
            ctx = ctx_for(B)
            A_b, E_b = _prefix(A, Bmax, B, bits), _prefix(E, Bmax, B, bits)
            Y_b = torch.zeros_like(A_b)
            for w in windows:
                mp.tune_set(bits, G, M, w)
                ws = torch.empty(mp.modexp_workspace_bytes(B, bits, w) // 4, dtype=torch.int32, device="cuda")
                ms = _time(lambda: mp.modexp_consttime(Y_b, A_b, E_b, bits, ctx, 0, workspace=ws))
                rate = B / (ms / 1e3)
                timings[f"modexp_G{G}_M{M}_w{w}"] = rate
                if log:
                    log(f"tune {bits}: G={G} M={M} w={w} batch={B}: {rate:,.0f} modexp/s")
                if best is None or rate > best[0]:
                    best = (rate, G, M, w)
        _, G, M, w = best
        mp.tune_set(bits, G, M, w)
        # window tables in shared memory (chosen shape), at the windows where they fit
        table = "global"
        for wt in windows:
            try:
                r = mp.table_residency(bits, wt)
            except mp.MpError:
                r = 0
            if r <= 0:
                continue
            B = rounds * sms * r
            ctx = ctx_for(B) if B <= Bmax else None
            if ctx is None:
                continue
            A_b, E_b = _prefix(A, Bmax, B, bits), _prefix(E, Bmax, B, bits)
            Y_b = torch.zeros_like(A_b)
            ws = torch.empty(mp.modexp_workspace_bytes(B, bits, wt) // 4, dtype=torch.int32, device="cuda")
            mp.tune_set_table(bits, mp.TABLE_SHARED)
            try:
                ms = _time(lambda: mp.modexp_consttime(Y_b, A_b, E_b, bits, ctx, wt, workspace=ws))
            finally:
                mp.tune_set_table(bits, mp.TABLE_GLOBAL)
            rate = B / (ms / 1e3)
            timings[f"modexp_shared_table_w{wt}"] = rate
            if log:
                log(f"tune {bits}: shared-memory tables w={wt} batch={B} ({r}/SM): {rate:,.0f} modexp/s")
            if rate > best[0]:
                best = (rate, G, M, wt)
                table = "shared"
        w = best[3]
        mp.tune_set(bits, G, M, w)
        mp.tune_set_table(bits, mp.TABLE_SHARED if table == "shared" else mp.TABLE_GLOBAL)
        # Montgomery products in the truncated Karatsuba form (Sec. 5.1) against the best choice
        mont_kara = NEVER
        if per_sm_tk:
            B = rounds * sms * per_sm_tk
            ctx = ctx_for(B)
            A_b, E_b = _prefix(A, Bmax, B, bits), _prefix(E, Bmax, B, bits)
            Y_b = torch.zeros_like(A_b)
            ws = torch.empty(mp.modexp_workspace_bytes(B, bits, w) // 4, dtype=torch.int32, device="cuda")
            ms = _time(lambda: mp.modexp_consttime(Y_b, A_b, E_b, bits, ctx, w, mp.RED_TRUNCATED, mp.ALGO_KARATSUBA,
                                                   workspace=ws))
            rate = B / (ms / 1e3)
            timings[f"modexp_karatsuba_form_w{w}"] = rate
            if log:
                log(f"tune {bits}: truncated Karatsuba form w={w} batch={B}: {rate:,.0f} modexp/s")
            if rate > best[0]:
                mont_kara = bits
        # products: schoolbook vs Karatsuba with the chosen shape
        n = (bits + 31) // 32
        B = Bmax
        C = torch.zeros(mp.array_words(IL, B, 2 * n), dtype=torch.int32, device="cuda")
        prod = {}
        for algo, nm in ((mp.ALGO_SCHOOLBOOK, "schoolbook"), (mp.ALGO_KARATSUBA, "karatsuba")):
            try:
                ms = _time(lambda: mp.mp_mul(C, A, E, B, bits, IL, algo), 3)
                prod[nm] = B / (ms / 1e3)
            except mp.MpError:
                prod[nm] = 0.0
        timings.update({f"mul_{k}": v for k, v in prod.items()})
        kara = prod["karatsuba"] > prod["schoolbook"]
        out[str(bits)] = {"G": G, "M": M, "window": w, "table": table, "karatsuba_from_bits": bits if kara else NEVER,
                          "mont_karatsuba_from_bits": mont_kara, "modexp_per_s": best[0],
                          "residency_per_sm": {f"G{g}_M{m}": r for (g, m), r in per_sm.items()}, "timings": timings}
        for c in ctxs.values():
            c.free()
    return out


def _prefix(X: torch.Tensor, batch: int, B: int, bits: int) -> torch.Tensor:
    """The first B instances of an interleaved device array of `batch` instances."""
    if B == batch:
        return X
    n = (bits + 31) // 32
    return mp.to_device(mp.interleave(mp.deinterleave(mp.to_host(X), batch, n)[:B]))


def apply(choice: dict):
    for bits, c in choice.items():
        mp.tune_set(int(bits), c["G"], c["M"], c["window"], c["karatsuba_from_bits"])
        mp.tune_set_table(int(bits), mp.TABLE_SHARED if c.get("table") == "shared" else mp.TABLE_GLOBAL)
        k = c.get("mont_karatsuba_from_bits", NEVER)
        mp.tune_set_mont_karatsuba(int(bits), 0 if k == NEVER else k)


def load_or_tune(sizes=(1024, 2048, 3072, 4096), path: str = CACHE, force: bool = False, log=None) -> dict:
    """Apply the cached choice for this GPU, tuning (and caching) the sizes it lacks."""
    key = _key()
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    entry = cache.get(key, {})
    todo = [b for b in sizes if force or str(b) not in entry]
    if todo:
        entry.update(tune(todo, log=log))
        cache[key] = entry
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    choice = {b: entry[b] for b in map(str, sizes)}
    apply(choice)
    return choice
