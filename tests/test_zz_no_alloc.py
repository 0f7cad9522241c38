"""modexp_consttime_noalloc: the exponentiation for callers that cannot allocate
device memory (its window tables sit in a fixed static array of the library).
Its results must equal those of modexp_consttime (with a caller workspace), bit
for bit, on two calls in a row with different inputs. Collected last on purpose."""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

IL = 1


def _run_pair(mp, bits, batch, window, sub, red=0, algo=0):
    b = si.make_batch(0, "test", batch, bits, sub=sub)
    dev = lambda x: mp.to_device(mp.interleave(x))
    ctx = mp.MontCtx(dev(b.N), batch, bits, IL)
    A, E = dev(b.a), dev(b.e)
    ws = torch.empty(mp.modexp_workspace_bytes(batch, bits, window) // 4, dtype=torch.int32, device="cuda")
    y_ref = torch.zeros_like(A)
    y_new = torch.full_like(A, -1)
    mp.modexp_consttime(y_ref, A, E, b.ebits, ctx, window, red, algo, workspace=ws)
    mp.modexp_consttime_noalloc(y_new, A, E, b.ebits, ctx, window, red, algo)
    torch.cuda.synchronize()
    got = mp.deinterleave(mp.to_host(y_new), batch, b.n)
    want = mp.deinterleave(mp.to_host(y_ref), batch, b.n)
    ctx.free()
    return got, want


# (reduction, product form): the truncated schoolbook kernels, the word-serial reduction
# (lane-mapped kernels) and the truncated Karatsuba form (its own kernels)
FORMS = [(0, 0), (2, 0), (0, 2)]


@pytest.mark.parametrize("red,algo", FORMS)
def test_noalloc_matches_workspace_version_on_two_calls(red, algo):
    import paper_2410_18129_gb300 as mp
    # first call: 2048-bit, w=5; second call: different size, batch and window, so a
    # second call that reused stale table contents would show up as a mismatch
    for bits, batch, window, sub in ((2048, 300, 5, 901), (1024, 700, 4, 902)):
        got, want = _run_pair(mp, bits, batch, window, sub, red, algo)
        bad = np.nonzero((got != want).any(axis=1))[0]
        assert bad.size == 0, f"{bits}-bit: {bad.size} instances differ, first {bad[:8]}"


def test_noalloc_rejects_batches_beyond_its_scratch():
    import paper_2410_18129_gb300 as mp
    bits, window = 2048, 5
    batch = mp.NOALLOC_SCRATCH_BYTES // (32 * 64 * 4) + 1     # one instance more than fits
    N = si.random_odd_moduli(si.stream(0, "test", "modulus", 903), batch, bits)
    dev = lambda x: mp.to_device(mp.interleave(x))
    ctx = mp.MontCtx(dev(N), batch, bits, IL)
    y = torch.zeros(batch * 64, dtype=torch.int32, device="cuda")
    with pytest.raises(mp.MpError) as e:
        mp.modexp_consttime_noalloc(y, y, y, bits, ctx, window)
    assert e.value.status == -2
    ctx.free()
