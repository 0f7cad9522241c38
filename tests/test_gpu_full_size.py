"""The 4096-bit workload (16384 instances at 4096 bits, w = 6, with its 4108-bit schoolbook
and 4154-bit Karatsuba product edges) and the mixed-size workload (100,000 exponentiations:
40 % 2048, 25 % 1024, 20 % 3072, 15 % 4096 bits) at their full sizes, in the launch
configurations bench.py times, checked against the oracle on sampled instances (exact
integers, tolerance 0)."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
IL = 1


def test_4096_bit_workload_at_size():
    import paper_2410_18129_gb300 as mp
    B = 16384
    dev = lambda x: mp.to_device(mp.interleave(x))
    idx = np.linspace(0, B - 1, 8).astype(int)
    for bits, algo in ((4108, mp.ALGO_SCHOOLBOOK), (4154, mp.ALGO_KARATSUBA)):
        b = si.batch_4096(0, B, bits)
        C = torch.zeros(mp.array_words(IL, B, 2 * b.n), dtype=torch.int32, device="cuda")
        mp.mp_mul(C, dev(b.a), dev(b.b), B, bits, IL, algo)
        got = mp.deinterleave(mp.to_host(C), B, 2 * b.n)[idx]
        assert np.array_equal(got, oracle.mul(b.a[idx], b.b[idx])), f"{bits}-bit products"
    b = si.batch_4096(0, B, 4096)
    N, A, Bv, E = (dev(x) for x in (b.N, b.a, b.b, b.e))
    ctx = mp.MontCtx(N, B, 4096, IL)
    C = torch.zeros_like(A)
    mp.mont_mul(C, A, Bv, ctx, mp.RED_TRUNCATED)
    got = mp.deinterleave(mp.to_host(C), B, b.n)[idx]
    assert np.array_equal(got, oracle.mont_def(b.a[idx], b.b[idx], b.N[idx])), "4096-bit Montgomery products"
    ws = torch.empty(mp.modexp_workspace_bytes(B, 4096, 6) // 4, dtype=torch.int32, device="cuda")
    Y = torch.zeros_like(A)
    mp.modexp_consttime(Y, A, E, b.ebits, ctx, 6, mp.RED_TRUNCATED, workspace=ws)
    got = mp.deinterleave(mp.to_host(Y), B, b.n)[idx]
    assert np.array_equal(got, oracle.modexp(b.a[idx], b.e[idx], b.ebits, b.N[idx])), "4096-bit exponentiations"
    ctx.free()


def test_mixed_workload_at_size():
    import paper_2410_18129_gb300 as mp
    total = 100000
    sizes = si.mixed_sizes(0, total)
    classes = [(bits, int((sizes == bits).sum())) for bits in (4096, 3072, 2048, 1024)]
    dev = lambda x: mp.to_device(mp.interleave(x))
    jobs, batches = [], []
    for bits, cnt in classes:
        b = si.make_batch(0, "mixed", cnt, bits, sub=bits)
        ctx = mp.MontCtx(dev(b.N), cnt, bits, IL)
        A, E = dev(b.a), dev(b.e)
        jobs.append((torch.zeros_like(A), A, E, bits, ctx, 0))
        batches.append(b)
    mp.modexp_consttime_mixed(jobs, mp.RED_TRUNCATED, mp.mixed_workspace(jobs))
    torch.cuda.synchronize()
    for (Y, A, E, bits, ctx, w), b in zip(jobs, batches):
        idx = np.linspace(0, b.batch - 1, 6).astype(int)
        got = mp.deinterleave(mp.to_host(Y), b.batch, b.n)[idx]
        assert np.array_equal(got, oracle.modexp(b.a[idx], b.e[idx], b.ebits, b.N[idx])), f"{bits}-bit class"
        ctx.free()
