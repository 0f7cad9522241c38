"""Benchmark: 2048-bit constant-time modexp/s (and Montmul/s) on GB300.

One step = one modexp_consttime call over the whole batch (65536 instances of
2048-bit moduli, half random odd and half products of two 1024-bit primes;
uniform bases; full-length 2048-bit exponents; window 5; truncated Montgomery;
interleaved layout): to-Montgomery conversion, window table, 410 windows of 5
squarings + a masked table scan + a product, and the conversion back.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun every rank runs its own batch
(weak scaling, no collective on the data path); `value` = all instances of all
ranks / the slowest rank's time. `--impl reference` times the CPU oracle (plain
left-to-right square-and-multiply) on a bounded sample of the same workload.

Beside the headline the default line carries, each with its fraction of the
measured IMAD roofline: the classical (Alg. 5) and word-serial (Alg. 4)
reductions on the same batch, the batched form (`mixed`: 100,000 exponentiations
of four sizes in one mixed call, plain one-launch-per-size and CUDA-graph end to
end beside it) and the served form (`serving`: Poisson arrivals at 1e4, 1e5 and
1e6 requests/s over a resident pool, p50/p99 latency, plain path beside it).
Every instance of the headline run is checked against the oracle on the host
cores while the GPU measures those forms (`parity`).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2048-bit const-time modexp/s and Montmul/s on 1 GB300; p99 latency under load"
BITS, WINDOW = 2048, 5


def imad_counts(n: int):
    """Algorithmic 32-bit multiply-add count (each partial product = a lo and a hi
    multiply-add) of one Montgomery product / square, truncated (Alg. 6) and full (Alg. 5)."""
    return {
        "mul_trunc": 4 * n * n + 2 * n - 1,
        "sqr_trunc": 3 * n * n + 3 * n - 1,
        "mul_full": 5 * n * n,
        "sqr_full": 4 * n * n + n,
    }


def modexp_imad(bits: int, ebits: int, w: int, red: str = "trunc") -> int:
    n = (bits + 31) // 32
    c = imad_counts(n)
    windows = (ebits + w - 1) // w
    sqrs = windows * w
    muls = windows + 1 + ((1 << w) - 2) + 1     # windows, to-Montgomery, table, from-Montgomery
    return sqrs * c["sqr_" + red] + muls * c["mul_" + red]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_rate(b, ebits, budget_s: float, threads: int = 0):
    """Time the CPU oracle's modexp on a sample of the workload sized for ~budget_s."""
    import oracle
    cores = oracle.threads_used(threads)
    k = max(cores, 8)
    t0 = time.perf_counter()
    oracle.modexp(b.a[:k], b.e[:k], ebits, b.N[:k], threads)
    dt = time.perf_counter() - t0
    count = int(min(b.batch, max(k, k * budget_s / max(dt, 1e-6))))
    t0 = time.perf_counter()
    oracle.modexp(b.a[:count], b.e[:count], ebits, b.N[:count], threads)
    dt = time.perf_counter() - t0
    return count / dt, cores, count, dt


def _load_replicas():
    """The replica helpers, loaded by path (they need no CUDA library)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "mpgpu_replicas", os.path.join(ROOT, "paper_2410_18129_gb300", "replicas.py"))
    mod = importlib.util.module_from_spec(spec)
    sys.modules["mpgpu_replicas"] = mod
    spec.loader.exec_module(mod)
    return mod


def sources_digest() -> str:
    """Digest of the CUDA sources and the C header: a recorded ncu figure applies only to the
    kernel built from exactly these sources."""
    import glob
    import hashlib
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(ROOT, "paper_2410_18129_gb300", "csrc", "*.cu*")) +
                   glob.glob(os.path.join(ROOT, "paper_2410_18129_gb300", "csrc", "*.h")) +
                   glob.glob(os.path.join(ROOT, "include", "*.h")))
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, instances: int):
    """DRAM bytes (read + write) per launch from profiles/traffic.json, scaled to `instances`;
    None when there is no record or the kernel sources changed since it was taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("sources_digest") != sources_digest():
        return None
    return rec["dram_bytes_per_launch"] * instances / rec["instances"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--quick", action="store_true",
                    help="time the modexp steps only (no comparison runs, no e2e, no CPU baseline): for profiling")
    ap.add_argument("--reduction", default="truncated", choices=["truncated", "full", "cios"],
                    help="reduction of the timed modexp steps with --quick (profiling); the full line "
                         "always times the truncated one and reports the others beside it")
    ap.add_argument("--algo", default="auto", choices=["auto", "karatsuba"],
                    help="product form of the timed modexp steps with --quick: karatsuba runs every "
                         "Montgomery product in the truncated Karatsuba form")
    ap.add_argument("--sampled-parity", action="store_true",
                    help="check 24 sampled instances against the oracle instead of all of them")
    ap.add_argument("--no-forms", action="store_true",
                    help="leave out the mixed-size and serving forms of the default line")
    ap.add_argument("--workload", default="batch_2048", choices=["batch_2048", "batch_4096", "mixed", "serving"],
                    help="batch_2048: the headline line; batch_4096: 4096-bit products (schoolbook vs "
                         "Karatsuba, 4108/4154 edges), Montgomery and w=6 modexp")
    args = ap.parse_args()
    if args.workload == "batch_4096":
        return bench_4096(args)
    if args.workload == "mixed":
        return bench_mixed(args)
    if args.workload == "serving":
        return bench_serving(args)

    reps = _load_replicas()
    info = reps.rank_info()
    world, rank, local = info.world, info.rank, info.local

    import numpy as np
    import seeded_inputs as si

    procs = min(16, os.cpu_count() or 1)
    # inputs are generated before any CUDA call (the prime pool uses spawned workers)
    b = si.batch_2048(seed=reps.rank_seed(0, rank), batch=args.batch, procs=procs)
    ebits = b.ebits

    if args.impl == "reference":
        if rank != 0:
            return
        steps_rates = []
        for s in range(args.warmup + args.steps):
            rate, cores, count, dt = cpu_oracle_rate(b, ebits, budget_s=max(2.0, 60.0 / (args.warmup + args.steps)))
            if s >= args.warmup:
                steps_rates.append((rate, cores, count, dt))
        rate = statistics.median(r[0] for r in steps_rates)
        cores, count = steps_rates[0][1], steps_rates[0][2]
        line = {
            "impl": "reference", "metric": METRIC, "value": rate, "unit": "modexp/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(r[3] for r in steps_rates),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "batch_2048: 2048-bit moduli (half RSA-like), 2048-bit exponents, w=5",
                       "batch": args.batch, "bits": BITS, "window": WINDOW},
            "cpu_baseline": {"value": rate, "unit": "modexp/s", "cores": cores, "kind": "oracle",
                             "sample": f"{count} instances per step of the 65536-instance workload"},
            "e2e": {"value": rate, "unit": "modexp/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0,
        }
        print(json.dumps(line))
        return

    import torch
    import paper_2410_18129_gb300 as mp

    reps.init(info)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    IL = mp.LAYOUT_INTERLEAVED
    B = args.batch
    n = b.n
    N = mp.to_device(mp.interleave(b.N))
    A = mp.to_device(mp.interleave(b.a))
    Bv = mp.to_device(mp.interleave(b.b))
    E = mp.to_device(mp.interleave(b.e))
    Y = torch.zeros_like(A)
    ctx = mp.MontCtx(N, B, BITS, IL)
    ws = torch.empty(mp.modexp_workspace_bytes(B, BITS, WINDOW) // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        reps.barrier(info)
        torch.cuda.synchronize()

    quick_red = {"truncated": mp.RED_TRUNCATED, "full": mp.RED_FULL, "cios": mp.RED_CIOS}[args.reduction]
    quick_algo = {"auto": mp.ALGO_AUTO, "karatsuba": mp.ALGO_KARATSUBA}[args.algo]
    if not args.quick and (quick_red != mp.RED_TRUNCATED or quick_algo != mp.ALGO_AUTO):
        raise SystemExit("--reduction and --algo apply to --quick runs only")

    def step(red=quick_red, algo=quick_algo):
        mp.modexp_consttime(Y, A, E, ebits, ctx, WINDOW, red, algo, workspace=ws)

    def timed(fn, k):
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        barrier()
        return reps.max_over_ranks(info, e0.elapsed_time(e1), device=dev)

    # roofline denominator: measured integer multiply-add rate per SM per clock
    imad_rate, imad_mhz = mp.bench_imad(0, 2000)
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count

    for _ in range(args.warmup):
        step()
    # parity spot check of this run's output (sampled instances vs the oracle), outside timing
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms = timed(step, args.steps)
    clocks = clk.summary()
    ms_step = ms / args.steps
    value = reps.job_rate(info, B, ms_step)

    if args.quick:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "modexp/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                              "quick": True, "reduction": args.reduction, "algo": args.algo, "batch_per_gpu": B,
                              "clocks": clocks}))
        ctx.free()
        return

    # classical reduction for comparison
    for _ in range(1):
        step(mp.RED_FULL)
    ms_full = timed(lambda: step(mp.RED_FULL), max(2, args.steps // 2)) / max(2, args.steps // 2)
    # word-serial CIOS (Alg. 4) for comparison
    step(mp.RED_CIOS)
    ms_cios = timed(lambda: step(mp.RED_CIOS), max(2, args.steps // 2)) / max(2, args.steps // 2)
    # truncated reduction in its Karatsuba form (Sec. 5.1) for comparison
    def step_tk():
        mp.modexp_consttime(Y, A, E, ebits, ctx, WINDOW, mp.RED_TRUNCATED, mp.ALGO_KARATSUBA, workspace=ws)
    step_tk()
    ms_tk = timed(step_tk, max(2, args.steps // 2)) / max(2, args.steps // 2)
    Y_tk = Y.clone()

    # Montgomery products over the same batch
    C = torch.zeros_like(A)
    mm = {}
    for red, algo, nm in ((mp.RED_TRUNCATED, mp.ALGO_AUTO, "trunc"), (mp.RED_FULL, mp.ALGO_AUTO, "full"),
                          (mp.RED_CIOS, mp.ALGO_AUTO, "cios"), (mp.RED_TRUNCATED, mp.ALGO_KARATSUBA, "tkara")):
        for _ in range(3):
            mp.mont_mul(C, A, Bv, ctx, red, algo)
        k = 50
        mm[nm] = world * B / (timed(lambda: mp.mont_mul(C, A, Bv, ctx, red, algo), k) / k / 1e3)
        for _ in range(3):
            mp.mont_sqr(C, A, ctx, red, algo)
        mm[nm + "_sqr"] = world * B / (timed(lambda: mp.mont_sqr(C, A, ctx, red, algo), k) / k / 1e3)

    # end to end through the C ABI with host buffers: H2D inputs, modexp, D2H result
    hA = torch.from_numpy(mp.interleave(b.a).view(np.int32)).pin_memory()
    hE = torch.from_numpy(mp.interleave(b.e).view(np.int32)).pin_memory()
    hY = torch.empty(Y.numel(), dtype=torch.int32).pin_memory()
    dA, dE = torch.empty_like(A), torch.empty_like(E)

    def e2e_step():
        dA.copy_(hA, non_blocking=True)
        dE.copy_(hE, non_blocking=True)
        mp.modexp_consttime(Y, dA, dE, ebits, ctx, WINDOW, mp.RED_TRUNCATED, workspace=ws)
        hY.copy_(Y, non_blocking=True)

    e2e_step()
    ms_e2e = timed(e2e_step, args.steps) / args.steps
    torch.cuda.synchronize()
    tk_same = bool(torch.equal(Y_tk, Y))   # every instance: Karatsuba form == schoolbook truncated
    h2d = (hA.numel() + hE.numel()) * 4
    d2h = hY.numel() * 4

    got_all = mp.deinterleave(mp.to_host(Y), B, n)   # this run's results, every instance

    traffic = recorded_traffic("k_modexp_2048_w5", B)
    imad = modexp_imad(BITS, ebits, WINDOW, "trunc")
    achieved = imad * B / (ms_step / 1e3) / 1e12
    peak = imad_peak(sms, imad_rate)
    peak_clock = peak * 1e12 / (sms * imad_rate * 1e6)
    obs_clock = clocks["sm_mhz"] or imad_mhz
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TIMAD/s", "frac": achieved / peak,
                "traffic": traffic,
                "traffic_unit": "bytes per launch (DRAM read + write, ncu, same kernel sources)",
                "peak_basis": f"{sms} SMs x {imad_rate:.1f} IMAD/clk/SM (measured) x {peak_clock:.0f} MHz max clock",
                "frac_at_observed_clock": achieved / (sms * imad_rate * obs_clock * 1e6 / 1e12),
                "imad_per_modexp": imad}

    cpu = None
    if rank == 0 and world == 1:
        rate, cores, count, dt = cpu_oracle_rate(b, ebits, args.cpu_budget)
        cpu = {"value": rate, "unit": "modexp/s", "cores": cores, "kind": "oracle",
               "sample": f"{count} of the 65536 instances ({dt:.1f} s), plain square-and-multiply"}

    # parity of the timed configuration: every instance against the oracle, in a host thread
    # (the oracle's native call releases the interpreter) while the GPU measures the batched
    # and served forms; on rank 0 only, two cores left to the serving loop
    parity = None
    checker = None
    if rank == 0:
        import oracle
        box = {}
        full = not args.sampled_parity
        idx = np.arange(B) if full else np.linspace(0, B - 1, 24).astype(int)
        threads = max(1, (os.cpu_count() or 2) - 2)

        def check():
            t0 = time.perf_counter()
            want = oracle.modexp(b.a[idx], b.e[idx], ebits, b.N[idx], threads)
            box["mismatches"] = int((got_all[idx] != want).any(axis=1).sum())
            box["seconds"] = time.perf_counter() - t0
        checker = threading.Thread(target=check, daemon=True)
        checker.start()

    # the batched (mixed sizes) and served forms, with their roofline fractions
    mixed = serving = None
    if rank == 0 and world == 1 and not args.no_forms:
        mixed = run_mixed(max(2, args.steps // 4), 2, 100000, peak)
        serving = run_serving((1e4, 1e5, 1e6), seconds=10.0, min_requests=100000, peak=peak)
    if checker is not None:
        checker.join()
        parity = {"checked": int(idx.size), "mismatches": box["mismatches"],
                  "oracle_seconds": round(box["seconds"], 1), "oracle_threads": threads,
                  "kind": "every instance" if full else "sampled"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "modexp/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "batch_2048: 65536 x 2048-bit moduli (half random odd, half p*q of 1024-bit "
                                   "primes), uniform bases, 2048-bit exponents, window 5, truncated Montgomery",
                       "batch_per_gpu": B, "bits": BITS, "window": WINDOW, "layout": "interleaved",
                       "l2": "working set (window tables 512 MiB + contexts) larger than L2",
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": world * B / (ms_e2e / 1e3), "unit": "modexp/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "modexp_full_reduction_per_s": world * B / (ms_full / 1e3),
            "modexp_cios_per_s": world * B / (ms_cios / 1e3),
            "modexp_tkara_per_s": world * B / (ms_tk / 1e3),
            "tkara_equals_schoolbook": tk_same,
            "montmul_per_s": {"trunc": mm["trunc"], "full": mm["full"], "cios": mm["cios"], "tkara": mm["tkara"]},
            "montsqr_per_s": {"trunc": mm["trunc_sqr"], "full": mm["full_sqr"], "cios": mm["cios_sqr"],
                              "tkara": mm["tkara_sqr"]},
            "parity": parity,
            "imad_microbench": {"per_clk_per_sm": imad_rate, "implied_mhz": imad_mhz},
            "mixed": mixed,
            "serving": serving,
        }
        print(json.dumps(line))
    ctx.free()
    if world > 1:
        torch.distributed.destroy_process_group()


def _event_timer(torch, stream):
    def timed(fn, k):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k
    return timed


def bench_4096(args):
    """4096-bit workload (16384 instances): products schoolbook vs one-level Karatsuba, the
    4108-bit (schoolbook) and 4154-bit (Karatsuba) edge sizes, truncated Montgomery products and
    the w=6 constant-time modexp. One JSON line; `value` is 4096-bit modexp/s."""
    import numpy as np
    import seeded_inputs as si
    import torch
    import paper_2410_18129_gb300 as mp
    import oracle

    B = 16384 if args.batch == 65536 else args.batch
    IL = mp.LAYOUT_INTERLEAVED
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    timed = _event_timer(torch, stream)
    out = {}
    prod = {}
    for bits in (4096, 4108, 4154):
        b = si.batch_4096(0, B, bits)
        n = b.n
        A, Bv = mp.to_device(mp.interleave(b.a)), mp.to_device(mp.interleave(b.b))
        C = torch.zeros(mp.array_words(IL, B, 2 * n), dtype=torch.int32, device="cuda")
        for algo, nm in ((mp.ALGO_SCHOOLBOOK, "schoolbook"), (mp.ALGO_KARATSUBA, "karatsuba"),
                         (mp.ALGO_KARATSUBA2, "karatsuba2")):
            for op in ("mul", "sqr"):
                f = (lambda: mp.mp_mul(C, A, Bv, B, bits, IL, algo)) if op == "mul" else \
                    (lambda: mp.mp_sqr(C, A, B, bits, IL, algo))
                for _ in range(args.warmup):
                    f()
                ms = timed(f, max(50, args.steps))   # a launch is tens of microseconds: time many
                prod[f"{op}_{nm}_{bits}"] = B / (ms / 1e3)
                # bit-exact spot check against the oracle
                got = mp.deinterleave(mp.to_host(C), B, 2 * n)[:16]
                want = oracle.mul(b.a[:16], b.b[:16]) if op == "mul" else oracle.sqr(b.a[:16])
                assert np.array_equal(got, want), (op, nm, bits)
    out["products_per_s"] = prod
    b = si.batch_4096(0, B, 4096)
    n = b.n
    N, A, Bv, E = (mp.to_device(mp.interleave(x)) for x in (b.N, b.a, b.b, b.e))
    ctx = mp.MontCtx(N, B, 4096, IL)
    C = torch.zeros_like(A)
    mm = {}
    for red, algo, nm in ((mp.RED_TRUNCATED, mp.ALGO_AUTO, "trunc"), (mp.RED_FULL, mp.ALGO_AUTO, "full"),
                          (mp.RED_TRUNCATED, mp.ALGO_KARATSUBA, "tkara")):
        for _ in range(3):
            mp.mont_mul(C, A, Bv, ctx, red, algo)
        mm["mul_" + nm] = B / (timed(lambda: mp.mont_mul(C, A, Bv, ctx, red, algo), 20) / 1e3)
        mm["sqr_" + nm] = B / (timed(lambda: mp.mont_sqr(C, A, ctx, red, algo), 20) / 1e3)
    out["mont_per_s"] = mm
    ws = torch.empty(mp.modexp_workspace_bytes(B, 4096, 6) // 4, dtype=torch.int32, device="cuda")
    Y = torch.zeros_like(A)
    step = lambda: mp.modexp_consttime(Y, A, E, b.ebits, ctx, 6, mp.RED_TRUNCATED, workspace=ws)
    for _ in range(args.warmup):
        step()
    with ClockSampler(0) as clk:
        ms = timed(step, args.steps)
    idx = np.linspace(0, B - 1, 6).astype(int)
    got = mp.deinterleave(mp.to_host(Y), B, n)[idx]
    want = oracle.modexp(b.a[idx], b.e[idx], b.ebits, b.N[idx])
    # the same exponentiation with every product in the truncated Karatsuba form (Sec. 5.1)
    Y_sb = Y.clone()
    step_tk = lambda: mp.modexp_consttime(Y, A, E, b.ebits, ctx, 6, mp.RED_TRUNCATED, mp.ALGO_KARATSUBA, workspace=ws)
    step_tk()
    ms_tk = timed(step_tk, max(2, args.steps))
    out["modexp_tkara_per_s"] = B / (ms_tk / 1e3)
    torch.cuda.synchronize()
    out["tkara_equals_schoolbook"] = bool(torch.equal(Y, Y_sb))
    ctx.free()
    # lazy reduction (no final subtraction while 4N <= W^NP): 4606-bit moduli have the slack
    # in the 144-word shape, 4607-bit ones do not; same shape, same work otherwise
    lazy = {}
    BL = min(B, 8192)
    for lb in (4606, 4607):
        bl = si.make_batch(0, "lazy", BL, lb)
        Nl, Al, El = (mp.to_device(mp.interleave(x)) for x in (bl.N, bl.a, bl.e))
        cl = mp.MontCtx(Nl, BL, lb, IL)
        wsl = torch.empty(mp.modexp_workspace_bytes(BL, lb, 6) // 4, dtype=torch.int32, device="cuda")
        Yl = torch.zeros_like(Al)
        f = lambda: mp.modexp_consttime(Yl, Al, El, lb, cl, 6, mp.RED_TRUNCATED, workspace=wsl)
        f()
        lazy[f"modexp_{lb}_per_s"] = BL / (timed(f, 2) / 1e3)
        gl = mp.deinterleave(mp.to_host(Yl), BL, bl.n)[:4]
        assert np.array_equal(gl, oracle.modexp(bl.a[:4], bl.e[:4], lb, bl.N[:4])), lb
        cl.free()
    lazy["saving"] = lazy["modexp_4606_per_s"] / lazy["modexp_4607_per_s"] - 1.0
    out["lazy_reduction"] = lazy
    line = {
        "metric": "4096-bit const-time modexp/s (w=6) and 4096-bit product rates", "value": B / (ms / 1e3),
        "unit": "modexp/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"batch_4096: {B} x 4096-bit random odd moduli, full-length exponents, w=6; "
                               "products at 4096/4108/4154 bits", "batch": B},
        "clocks": clk.summary(), "parity": {"sampled": int(idx.size),
                                            "mismatches": int((got != want).any(axis=1).sum())},
        **out,
    }
    print(json.dumps(line))


def imad_peak(sms: int, imad_rate: float) -> float:
    """Roofline denominator in T IMAD/s: SMs x measured multiply-adds per SM per clock x the
    maximum SM clock (MEASURED_PEAKS.json when present)."""
    peak_clock = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak_clock = float(json.load(f).get("sm_max_mhz", peak_clock))
    except Exception:
        pass
    return sms * imad_rate * peak_clock * 1e6 / 1e12


def fixed_base_imad(bits: int, ebits: int, w: int) -> int:
    """Multiply-adds of one fixed-base request on a resident table (truncated reduction): the
    window loop and the product with 1, no table build and no conversion of the base."""
    c = imad_counts((bits + 31) // 32)
    windows = (ebits + w - 1) // w
    return windows * w * c["sqr_trunc"] + (windows + 1) * c["mul_trunc"]


def run_mixed(steps: int, warmup: int, total: int = 100000, peak: float | None = None, log=None):
    """Mixed sizes: `total` exponentiations, 40% 2048 / 25% 1024 / 20% 3072 / 15% 4096 bits,
    full-length exponents. The autotuner picks shape and window per size; three forms are
    timed: one launch per size (plain), the mixed call over all sizes (one launch per job on
    parallel streams, costliest first), and the mixed call replayed from a CUDA graph together
    with the host->device input copies and the result copies (end to end)."""
    import numpy as np
    import seeded_inputs as si
    import torch
    import paper_2410_18129_gb300 as mp
    from paper_2410_18129_gb300 import tune
    import oracle

    sizes = si.mixed_sizes(0, total)
    classes = [(bits, int((sizes == bits).sum())) for bits in (4096, 3072, 2048, 1024)]
    batches = {bits: si.make_batch(0, "mixed", cnt, bits, sub=bits) for bits, cnt in classes}
    stream = torch.cuda.current_stream()
    timed = _event_timer(torch, stream)
    choice = tune.load_or_tune(sizes=(1024, 2048, 3072, 4096))
    IL = mp.LAYOUT_INTERLEAVED
    dev = lambda x: mp.to_device(mp.interleave(x))
    jobs, ctxs, plain_ws, host = [], [], {}, []
    for bits, cnt in classes:
        b = batches[bits]
        ctx = mp.MontCtx(dev(b.N), cnt, bits, IL)
        A, E = dev(b.a), dev(b.e)
        Y = torch.zeros_like(A)
        jobs.append((Y, A, E, bits, ctx, 0))
        ctxs.append(ctx)
        w = choice[str(bits)]["window"]
        plain_ws[bits] = torch.empty(mp.modexp_workspace_bytes(cnt, bits, w) // 4, dtype=torch.int32, device="cuda")
        host.append((torch.from_numpy(mp.interleave(b.a).view(np.int32)).pin_memory(),
                     torch.from_numpy(mp.interleave(b.e).view(np.int32)).pin_memory(),
                     torch.empty(Y.numel(), dtype=torch.int32).pin_memory()))
    ws = mp.mixed_workspace(jobs)

    def plain():
        for (Y, A, E, bits, ctx, w), (_, cnt) in zip(jobs, classes):
            mp.modexp_consttime(Y, A, E, bits, ctx, 0, workspace=plain_ws[bits])

    def mixed():
        mp.modexp_consttime_mixed(jobs, mp.RED_TRUNCATED, ws)

    def e2e():
        for (Y, A, E, *_), (hA, hE, hY) in zip(jobs, host):
            A.copy_(hA, non_blocking=True)
            E.copy_(hE, non_blocking=True)
        mixed()
        for (Y, *_), (hA, hE, hY) in zip(jobs, host):
            hY.copy_(Y, non_blocking=True)

    for _ in range(warmup):
        plain()
        mixed()
        e2e()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        e2e()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    with torch.cuda.graph(graph):
        e2e()
    k = max(2, steps)
    ms_plain = timed(plain, k)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms_mixed = timed(mixed, k)
    ms_graph = timed(graph.replay, k)
    cios = lambda: mp.modexp_consttime_mixed(jobs, mp.RED_CIOS, ws)
    cios()
    ms_cios = timed(cios, k)
    # parity: each size class, sampled instances of the graph-replayed results vs the oracle
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    mism, sampled = 0, 0
    for (bits, cnt), (hA, hE, hY) in zip(classes, host):
        b = batches[bits]
        got = mp.deinterleave(hY.numpy().view(np.uint32), cnt, b.n)
        idx = np.linspace(0, cnt - 1, 6).astype(int)
        want = oracle.modexp(b.a[idx], b.e[idx], b.ebits, b.N[idx])
        mism += int((got[idx] != want).any(axis=1).sum())
        sampled += idx.size
    imad = sum(cnt * modexp_imad(bits, bits, choice[str(bits)]["window"], "trunc") for bits, cnt in classes)
    h2d = sum((hA.numel() + hE.numel()) * 4 for hA, hE, _ in host)
    d2h = sum(hY.numel() * 4 for *_, hY in host)

    def roof(ms):
        achieved = imad / (ms / 1e3) / 1e12
        return {"achieved": achieved, "frac": achieved / peak if peak else None}

    out = {
        "workload": f"mixed: {total} modexp, sizes " + ", ".join(f"{c} x {b}" for b, c in classes)
                    + " bits, random odd moduli, full-length exponents, truncated Montgomery",
        "modexp_per_s": total / (ms_mixed / 1e3), "ms_per_step": ms_mixed, "steps": k,
        "form": "one launch per job on parallel streams, costliest first",
        "plain_per_size_launches_per_s": total / (ms_plain / 1e3),
        "speedup_vs_plain": ms_plain / ms_mixed,
        "cios_mixed_per_s": total / (ms_cios / 1e3),
        "e2e": {"value": total / (ms_graph / 1e3), "unit": "modexp/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "form": "CUDA graph: H2D copies + mixed call + D2H copies"},
        "roofline": {"bound": "alu", "unit": "TIMAD/s", "peak": peak, "imad_per_step": imad,
                     **roof(ms_mixed), "plain": roof(ms_plain)},
        "tuned": {b: {k2: v for k2, v in c.items() if k2 != "timings"} for b, c in choice.items()},
        "clocks": clk.summary(), "parity": {"sampled": sampled, "mismatches": mism},
    }
    for c in ctxs:
        c.free()
    return out


def bench_mixed(args):
    """--workload mixed: the mixed-size forms on their own (one JSON line; `value` is the mixed
    call's modexp/s)."""
    import torch
    import paper_2410_18129_gb300 as mp
    torch.cuda.set_device(0)
    rate, _ = mp.bench_imad(0, 2000)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    total = 100000 if args.batch == 65536 else args.batch
    m = run_mixed(args.steps, args.warmup, total, imad_peak(sms, rate))
    line = {
        "metric": "mixed-size const-time modexp/s (mixed call; CUDA graph end to end)",
        "value": m["modexp_per_s"], "unit": "modexp/s", "n_gpus": 1, "steps": m["steps"], "warmup": args.warmup,
        "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic", "config": {"workload": m["workload"], "tuned": m["tuned"]},
        "e2e": m["e2e"], "roofline": m["roofline"], "gpu_launches": 4, "clocks": m["clocks"],
        "parity": m["parity"], "plain_per_size_launches_per_s": m["plain_per_size_launches_per_s"],
        "cios_mixed_per_s": m["cios_mixed_per_s"],
    }
    print(json.dumps(line))


def run_serving(rates=(1e4, 1e5, 1e6), seconds: float = 10.0, min_requests: int = 100000, cap: int = 400000,
                peak: float | None = None, plain: bool = True, variable_rates=(1e4, 1e5)):
    """Serving: Poisson arrivals over a resident pool of 4096 moduli (mixed sizes, fixed bases,
    tables on the device). Each rate runs for `seconds` of arrivals or `min_requests` requests,
    whichever is more (at most `cap`), through the continuous-batching loop (4 streams, one
    mixed call per batch, admission by device memory) and, for comparison, through the plain
    path (one batch at a time, one launch per size). Reports p50/p99 latency, throughput and
    the achieved fraction of the IMAD roofline of the served requests. The same loop then
    serves variable-base requests (each with its own base) at `variable_rates`."""
    import numpy as np
    import seeded_inputs as si
    import torch
    import paper_2410_18129_gb300 as mp
    from paper_2410_18129_gb300 import serve as sv
    from paper_2410_18129_gb300 import tune

    choice = tune.load_or_tune(sizes=(1024, 2048, 3072, 4096))
    pin = si.serving_pool(0, 4096)
    pool = sv.Pool(mp, pin.sizes, pin.moduli, pin.bases)
    # free device memory, counting what torch's allocator holds unused as free
    free_fn = lambda: torch.cuda.mem_get_info()[0] + torch.cuda.memory_reserved() - torch.cuda.memory_allocated()

    def run(tr, with_plain):
        bits = pool.sizes[tr.entry]
        var = [b is not None for b in tr.bases] if tr.bases is not None else [False] * len(bits)
        imad = 0
        for bb, v in zip(bits, var):
            bb = int(bb)
            w = pool.classes[bb]["window"]
            imad += modexp_imad(bb, bb, w, "trunc") if v else fixed_base_imad(bb, bb, w)
        adm = sv.AdmissionController(free_fn=free_fn, fraction=0.5, reserve=1 << 30, refresh=0.1)
        cont = sv.serve(tr, sv.ContinuousExecutor(pool, tr, slots=2), slots=2, max_batch=16384, admission=adm)
        cs = cont.summary()
        span = float(np.nanmax(cont.done_at))
        cs["roofline"] = {"achieved": imad / span / 1e12, "frac": imad / span / 1e12 / peak if peak else None,
                          "imad": imad}
        entry = {"requests": len(bits), "continuous": cs}
        if with_plain:
            entry["plain"] = sv.serve(tr, sv.PlainExecutor(pool, tr), slots=1, max_batch=16384).summary()
        return entry

    out, out_var = {}, {}
    with ClockSampler(torch.cuda.current_device()) as clk:
        for r in rates:
            count = int(min(cap, max(r * seconds, min_requests)))
            tr = si.poisson_trace(0, r, count, pool.sizes)
            out[f"{r:.0e}"] = {"offered_per_s": r, **run(tr, plain and r < 1e6)}
        for r in variable_rates:
            count = int(min(cap, max(r * seconds, min_requests)))
            tr = si.with_bases(si.poisson_trace(1, r, count, pool.sizes), pin, 1.0)
            out_var[f"{r:.0e}"] = {"offered_per_s": r, **run(tr, False)}
    res = {
        "workload": "serving: pool of 4096 moduli (1639 x 2048, 1024 x 1024, 819 x 3072, 614 x 4096 bits), fixed "
                    "base per modulus with resident tables, full-length exponents, Poisson arrivals, "
                    f">= {seconds:.0f} s or >= {min_requests} requests per rate",
        "windows": {b: c["window"] for b, c in choice.items()}, "slots": 2,
        "lanes": "one queue per size class, 2 batches in flight per class (a batch holds one class)",
        "max_batch": 16384,
        "rates": out, "variable_base_rates": out_var,
        "variable_base": "every request brings its own base: its window table (2^w - 2 more products) is built "
                         "per request", "clocks": clk.summary(),
    }
    pool.free()
    return res


def bench_serving(args):
    """--workload serving: the serving loop on its own (one JSON line; `value` is the continuous
    loop's throughput at the highest rate)."""
    import torch
    import paper_2410_18129_gb300 as mp
    torch.cuda.set_device(0)
    rate, _ = mp.bench_imad(0, 2000)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    res = run_serving((1e4, 3e4, 1e5, 3e5, 1e6), peak=imad_peak(sms, rate))
    top = res["rates"]["1e+06"]["continuous"]
    line = {
        "metric": "serving: p50/p99 latency and throughput under Poisson load (mixed sizes, resident moduli)",
        "value": top["throughput_per_s"], "unit": "modexp/s", "n_gpus": 1, "steps": len(res["rates"]), "warmup": 0,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": {k: v for k, v in res.items() if k not in ("rates", "clocks")},
        "rates": res["rates"], "clocks": res["clocks"],
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
