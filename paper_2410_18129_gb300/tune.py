"""Autotuner: per operand size, pick the group shape (threads per instance G x words per
thread M), the exponentiation window (4..6) and the schoolbook/Karatsuba choice for
products, by timing the library's own kernels on this GPU; apply the choice through
mp_tune_set and cache it as JSON keyed by GPU name, SM count and size.

    import paper_2410_18129_gb300.tune as tune
    choice = tune.load_or_tune(sizes=(1024, 2048, 3072, 4096))   # times, caches, applies

Timing: CUDA events on the current stream after one warm-up launch, full-length
exponents, a probe batch that fills every SM more than once.
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


def tune(sizes=(1024, 2048, 3072, 4096), windows=(4, 5, 6), batch: int | None = None, log=None):
    """Time every (shape, window) for each size and both product algorithms; returns the
    choice per size (not applied)."""
    IL = mp.LAYOUT_INTERLEAVED
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out = {}
    for bits in sizes:
        B = batch or 96 * sms * 2
        N, A, E = _probe(bits, B)
        ctx = mp.MontCtx(N, B, bits, IL)
        Y = torch.zeros_like(A)
        timings = {}
        best = None
        for G, M in mp.shape_candidates(bits):
            for w in windows:
                mp.tune_set(bits, G, M, w)
                ws = torch.empty(mp.modexp_workspace_bytes(B, bits, w) // 4, dtype=torch.int32, device="cuda")
                ms = _time(lambda: mp.modexp_consttime(Y, A, E, bits, ctx, 0, workspace=ws))
                rate = B / (ms / 1e3)
                timings[f"modexp_G{G}_M{M}_w{w}"] = rate
                if log:
                    log(f"tune {bits}: G={G} M={M} w={w}: {rate:,.0f} modexp/s")
                if best is None or rate > best[0]:
                    best = (rate, G, M, w)
        # products: schoolbook vs Karatsuba with the chosen shape
        _, G, M, w = best
        mp.tune_set(bits, G, M, w)
        n = (bits + 31) // 32
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
        out[str(bits)] = {"G": G, "M": M, "window": w, "karatsuba_from_bits": bits if kara else NEVER,
                          "modexp_per_s": best[0], "timings": timings}
        ctx.free()
    return out


def apply(choice: dict):
    for bits, c in choice.items():
        mp.tune_set(int(bits), c["G"], c["M"], c["window"], c["karatsuba_from_bits"])


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
