"""The mixed-size call captured in a CUDA graph together with its copies: host-to-device
copies of the inputs from pinned buffers, the mixed call (four sizes and one fixed-base
job), device-to-host copies of the results. The graph is replayed twice with new inputs
written into the same pinned buffers; every output word is compared with the oracle
(exact integers, tolerance 0)."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_mixed_call_replayed_from_a_cuda_graph():
    import paper_2410_18129_gb300 as mp
    IL = mp.LAYOUT_INTERLEAVED
    specs = [(4096, 9, 6), (3072, 11, 5), (2048, 30, 5), (1024, 45, 4)]
    fixed_bits, fixed_pool, nreq, fixed_w = 2048, 12, 20, 5
    # contexts and buffers are fixed across replays; inputs change
    ctxs, dev_in, pinned, moduli = [], [], [], []
    for k, (bits, batch, w) in enumerate(specs):
        b = si.make_batch(0, "mixed", batch, bits, sub=100 + k)
        moduli.append(b.N)
        ctxs.append(mp.MontCtx(mp.to_device(mp.interleave(b.N)), batch, bits, IL))
        hA = torch.empty(mp.array_words(IL, batch, b.n), dtype=torch.int32).pin_memory()
        hE = torch.empty_like(hA).pin_memory()
        hY = torch.empty_like(hA).pin_memory()
        pinned.append((hA, hE, hY))
        dev_in.append((torch.empty_like(hA, device="cuda"), torch.empty_like(hA, device="cuda"),
                       torch.zeros_like(hA, device="cuda")))
    # fixed-base job: a resident pool of moduli with their tables; requests carry (entry, exponent)
    fb = si.make_batch(0, "serving", fixed_pool, fixed_bits, ebits=1, sub=300)
    fctx = mp.MontCtx(mp.to_device(mp.interleave(fb.N)), fixed_pool, fixed_bits, IL)
    tables = torch.empty(mp.modexp_table_bytes(fctx, fixed_w) // 4, dtype=torch.int32, device="cuda")
    mp.modexp_table_build(tables, mp.to_device(mp.interleave(fb.a)), fctx, fixed_w)
    hIdx = torch.empty(nreq, dtype=torch.int32).pin_memory()
    hFE = torch.empty(mp.array_words(IL, nreq, fb.n), dtype=torch.int32).pin_memory()
    hFY = torch.empty_like(hFE).pin_memory()
    dIdx, dFE, dFY = (torch.empty_like(hIdx, device="cuda"), torch.empty_like(hFE, device="cuda"),
                      torch.zeros_like(hFE, device="cuda"))
    jobs = [(Y, A, E, bits, ctx, w) for (A, E, Y), ctx, (bits, _, w) in zip(dev_in, ctxs, specs)]
    jobs.append((dFY, None, dFE, fixed_bits, fctx, fixed_w, dIdx, tables, nreq))
    ws = mp.mixed_workspace(jobs)

    def fill(rep):
        """New inputs for replay `rep`, written into the pinned buffers; returns the oracle's results."""
        want = []
        for k, ((bits, batch, w), (hA, hE, hY), N) in enumerate(zip(specs, pinned, moduli)):
            a = si.uniform_below(si.stream(rep, "mixed", "base", 500 + k), N, bits)
            e = si.random_bits(si.stream(rep, "mixed", "exponent", 500 + k), batch, bits)
            hA.copy_(torch.from_numpy(mp.interleave(a).view(np.int32)))
            hE.copy_(torch.from_numpy(mp.interleave(e).view(np.int32)))
            want.append(oracle.modexp(a, e, bits, N))
        rng = si.stream(rep, "serving", "arrival", 301)
        idx = rng.integers(0, fixed_pool, size=nreq).astype(np.uint32)
        e = si.random_bits(si.stream(rep, "serving", "exponent", 302), nreq, fixed_bits)
        hIdx.copy_(torch.from_numpy(idx.view(np.int32)))
        hFE.copy_(torch.from_numpy(mp.interleave(e).view(np.int32)))
        want.append(oracle.modexp(fb.a[idx], e, fixed_bits, fb.N[idx]))
        return want

    def step():
        for (hA, hE, hY), (A, E, Y) in zip(pinned, dev_in):
            A.copy_(hA, non_blocking=True)
            E.copy_(hE, non_blocking=True)
        dIdx.copy_(hIdx, non_blocking=True)
        dFE.copy_(hFE, non_blocking=True)
        mp.modexp_consttime_mixed(jobs, mp.RED_TRUNCATED, ws)
        for (hA, hE, hY), (A, E, Y) in zip(pinned, dev_in):
            hY.copy_(Y, non_blocking=True)
        hFY.copy_(dFY, non_blocking=True)

    fill(0)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):   # warm-up outside the capture (creates the call's streams)
        step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for rep in (1, 2):
        want = fill(rep)
        for _, _, hY in pinned:
            hY.zero_()
        hFY.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for k, ((bits, batch, w), (_, _, hY)) in enumerate(zip(specs, pinned)):
            n = (bits + 31) // 32
            got = mp.deinterleave(hY.numpy().view(np.uint32), batch, n)
            assert np.array_equal(got, want[k]), f"replay {rep}: {bits}-bit job differs from the oracle"
        got = mp.deinterleave(hFY.numpy().view(np.uint32), nreq, fb.n)
        assert np.array_equal(got, want[-1]), f"replay {rep}: fixed-base job differs from the oracle"
    for c in ctxs + [fctx]:
        c.free()
