"""Serving loop on the GPU: every request served in a continuously batched launch gives the
same result as when it is computed alone and as the one-size-per-launch path; sampled
requests match the oracle. Fixed-base requests (resident tables) and variable-base requests
(their own base and table) are mixed in one trace. Tolerance 0 (exact integers)."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def request_base(pool, trace, r):
    """The base of request r: its own, or the fixed base of its pool entry."""
    if trace.bases is not None and trace.bases[r] is not None:
        return trace.bases[r]
    k = int(trace.entry[r])
    return pool.classes[int(pool.sizes[k])]["g"][int(pool.local[k])]


def expected(pool, trace, reqs):
    """Oracle results of the given requests: the request's base to its exponent mod the
    modulus of its pool entry."""
    out = {}
    for r in reqs:
        k = int(trace.entry[r])
        bits = int(pool.sizes[k])
        c = pool.classes[bits]
        j = int(pool.local[k])
        y = oracle.modexp(request_base(pool, trace, r)[None, :], trace.exponents[r][None, :], bits, c["N"][j:j + 1])
        out[int(r)] = y[0]
    return out


def test_served_results_equal_alone_and_plain():
    import paper_2410_18129_gb300 as mp
    from paper_2410_18129_gb300 import serve as sv
    pin = si.serving_pool(0, 96)
    pool = sv.Pool(mp, pin.sizes, pin.moduli, pin.bases, windows={1024: 4, 2048: 5, 3072: 5, 4096: 6})
    tr = si.with_bases(si.poisson_trace(0, 2e4, 360, pool.sizes), pin, 0.3)
    cont = sv.ContinuousExecutor(pool, tr, slots=3, keep_results=True)
    res = sv.serve(tr, cont, slots=3, max_batch=48,
                   admission=sv.AdmissionController(free_fn=lambda: torch.cuda.mem_get_info()[0]))
    assert len(res.results) == 360 and res.batches > 3
    plain = sv.PlainExecutor(pool, tr, keep_results=True)
    res_p = sv.serve(tr, plain, slots=1, max_batch=48)
    for r in range(360):
        assert np.array_equal(res.results[r], res_p.results[r]), r
    # alone: one request per launch
    IL = mp.LAYOUT_INTERLEAVED
    sizes = pool.sizes[tr.entry]
    sample = [r for r in range(360) if sizes[r] <= 2048][:12] + [r for r in range(360) if sizes[r] > 2048][:4]
    var = [r for r in range(360) if tr.bases[r] is not None]
    sample = sample + var[:6]
    for r in sample:
        bits = int(sizes[r])
        c = pool.classes[bits]
        y = torch.zeros(mp.array_words(IL, 1, c["n"]), dtype=torch.int32, device="cuda")
        idx = mp.to_device(np.array([pool.local[tr.entry[r]]], np.uint32))
        ex = mp.to_device(mp.interleave(tr.exponents[r][None, :]))
        if tr.bases[r] is None:
            mp.modexp_fixed_base(y, idx, ex, bits, 1, c["ctx"], c["tables"], c["window"])
        else:
            job = [(y, mp.to_device(mp.interleave(tr.bases[r][None, :])), ex, bits, c["ctx"], c["window"], idx, None, 1)]
            mp.modexp_consttime_mixed(job, mp.RED_TRUNCATED, mp.mixed_workspace(job))
        alone = mp.deinterleave(mp.to_host(y), 1, c["n"])[0]
        assert np.array_equal(alone, res.results[r]), r
    want = expected(pool, tr, sample)
    for r in sample:
        assert np.array_equal(want[r], res.results[r]), r
    pool.free()
