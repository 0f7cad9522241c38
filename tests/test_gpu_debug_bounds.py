"""The bounds-checking debug build (-DMPG_DEBUG_BOUNDS): its kernels check their shared-memory
block accesses, the instance and word offsets of their global loads and stores and their
window-table entries, record the first failed check and skip the access. Every entry point
family runs here on ragged batches in both layouts and agrees with the oracle, with no
violation recorded; the checks' own self-test records exactly one. The debug library runs in a
child process (MPGPU_LIB), so that this process keeps the release build."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu
pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent('''
    import numpy as np, torch
    import paper_2410_18129_gb300 as mp
    import oracle
    import seeded_inputs as si

    IM, IL = mp.LAYOUT_INSTANCE_MAJOR, mp.LAYOUT_INTERLEAVED
    torch.cuda.set_device(0)

    def dev(x, lay):
        return mp.to_device(mp.interleave(x) if lay == IL else np.ascontiguousarray(x).reshape(-1))

    def out(batch, w, lay):
        return torch.zeros(mp.array_words(lay, batch, w), dtype=torch.int32, device="cuda")

    def host(t, batch, w, lay):
        a = mp.to_host(t)
        return a.reshape(batch, w) if lay == IM else mp.deinterleave(a, batch, w)

    def same(got, want, what):
        if not np.array_equal(got, want):
            v = mp.debug_bounds()
            raise AssertionError(f"{what}: results differ; recorded violation kind {v >> 56}, "
                                 f"offset {v & ((1 << 56) - 1)}")

    assert mp.debug_bounds() == 0
    for bits in (1000, 1024, 2048, 3072, 4096, 4108):
        batch = 37
        b = si.make_batch(0, "test", batch, bits, ebits=40, sub=9100 + bits)
        n = b.n
        for lay in (IM, IL):
            A, B, N, E = dev(b.a, lay), dev(b.b, lay), dev(b.N, lay), dev(b.e, lay)
            C = out(batch, 2 * n, lay)
            algos = [mp.ALGO_SCHOOLBOOK, mp.ALGO_KARATSUBA] + ([mp.ALGO_KARATSUBA2] if bits >= 4096 else [])
            for algo in algos:
                mp.mp_mul(C, A, B, batch, bits, lay, algo)
                same(host(C, batch, 2 * n, lay), oracle.mul(b.a, b.b), f"mul {bits} {lay} {algo}")
                mp.mp_sqr(C, A, batch, bits, lay, algo)
                same(host(C, batch, 2 * n, lay), oracle.sqr(b.a), f"sqr {bits} {lay} {algo}")
            ctx = mp.MontCtx(N, batch, bits, lay)
            Y = out(batch, n, lay)
            want_m = oracle.mont_def(b.a, b.b, b.N)
            want_e = oracle.modexp(b.a, b.e, 40, b.N)
            for red in (mp.RED_TRUNCATED, mp.RED_FULL, mp.RED_CIOS):
                mp.mont_mul(Y, A, B, ctx, red)
                same(host(Y, batch, n, lay), want_m, f"mont_mul {bits} {lay} {red}")
                mp.modexp_consttime(Y, A, E, 40, ctx, 4, red)
                same(host(Y, batch, n, lay), want_e, f"modexp {bits} {lay} {red}")
            if bits <= 4096 and bits != 1000:
                mp.mont_mul(Y, A, B, ctx, mp.RED_TRUNCATED, mp.ALGO_KARATSUBA)
                same(host(Y, batch, n, lay), want_m, f"tkara mont_mul {bits} {lay}")
            if lay == IL:
                mp.modexp_consttime_noalloc(Y, A, E, 40, ctx, 4)
                same(host(Y, batch, n, lay), want_e, f"noalloc {bits}")
                mp.tune_set_table(bits, mp.TABLE_SHARED)
                try:
                    mp.modexp_consttime(Y, A, E, 40, ctx, 2)
                finally:
                    mp.tune_set_table(bits, mp.TABLE_GLOBAL)
                same(host(Y, batch, n, lay), want_e, f"shared tables {bits}")
                # resident fixed-base tables and routed requests
                w = 3
                tables = torch.empty(mp.modexp_table_bytes(ctx, w) // 4, dtype=torch.int32, device="cuda")
                mp.modexp_table_build(tables, A, ctx, w)
                idx = np.array([5, 0, 36, 5, 17], dtype=np.uint32)
                e_r = b.e[[1, 2, 3, 4, 6]]
                Yr = out(5, n, IL)
                mp.modexp_fixed_base(Yr, mp.to_device(idx.view(np.int32)), dev(e_r, IL), 40, 5, ctx, tables, w)
                same(host(Yr, 5, n, IL), oracle.modexp(b.a[idx.astype(np.int64)], e_r, 40, b.N[idx.astype(np.int64)]),
                     f"fixed base {bits}")
            ctx.free()
    # a mixed call over several classes (interleaved)
    jobs, keep = [], []
    for bits, batch in ((1024, 45), (2048, 40), (4096, 9)):
        b = si.make_batch(0, "test", batch, bits, ebits=32, sub=9300 + bits)
        ctx = mp.MontCtx(dev(b.N, IL), batch, bits, IL)
        Y = out(batch, b.n, IL)
        jobs.append((Y, dev(b.a, IL), dev(b.e, IL), 32, ctx, 0))
        keep.append((b, ctx))
    mp.modexp_consttime_mixed(jobs, mp.RED_TRUNCATED, mp.mixed_workspace(jobs))
    torch.cuda.synchronize()
    for (Y, *_), (b, ctx) in zip(jobs, keep):
        same(host(Y, b.batch, b.n, IL), oracle.modexp(b.a, b.e, 32, b.N), f"mixed {b.bits}")
        ctx.free()
    v = mp.debug_bounds()
    assert v == 0, f"bounds violation recorded: kind {v >> 56}, offset {v & ((1 << 56) - 1)}"
    mp.debug_bounds_selftest()
    v = mp.debug_bounds()
    assert v >> 56 == 6 and v & ((1 << 56) - 1) == 12345, hex(v)
    assert mp.debug_bounds() == 0
    print("debug bounds ok")
''')


def test_debug_build_records_no_violation():
    import __graft_entry__
    lib = __graft_entry__._load_build_script().build(debug=True)
    env = dict(os.environ, MPGPU_LIB=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0 and "debug bounds ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]


def test_release_build_has_no_checks():
    """The release library reports the debug entry points as not built."""
    import paper_2410_18129_gb300 as mp
    for f in (mp.debug_bounds, mp.debug_bounds_selftest):
        with pytest.raises(mp.MpError) as e:
            f()
        assert e.value.status == -7
