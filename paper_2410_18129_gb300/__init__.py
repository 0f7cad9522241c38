"""Python binding of libmpgpu (include/mpgpu.h): argument marshalling only.

Every function takes torch CUDA tensors of dtype int32/uint32 (any 32-bit integer
view), passes their device pointers and the current CUDA stream to the C ABI, and
raises MpError on a non-zero status. All arithmetic runs in the library's CUDA
kernels; there is no CPU fallback: importing on a machine without the built
library raises ImportError.

Names follow the C ABI: mp_mul, mp_sqr, mont_ctx_init (-> MontCtx), mont_mul,
mont_sqr, modexp_consttime, mp_convert.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# MPGPU_LIB: another build of the library (e.g. the bounds-checking debug build)
LIB_PATH = os.environ.get("MPGPU_LIB") or os.path.join(_HERE, "_build", "libmpgpu.so")

LAYOUT_INSTANCE_MAJOR, LAYOUT_INTERLEAVED = 0, 1
ALGO_AUTO, ALGO_SCHOOLBOOK, ALGO_KARATSUBA, ALGO_KARATSUBA2 = 0, 1, 2, 3
RED_TRUNCATED, RED_FULL, RED_CIOS = 0, 1, 2
TABLE_GLOBAL, TABLE_SHARED = 0, 1

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libmpgpu.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                      "or python paper_2410_18129_gb300/build.py")

_lib = ctypes.CDLL(LIB_PATH)
_vp, _sz, _u32, _i = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_int
_SIG = {
    "mp_strerror": ([_i], ctypes.c_char_p),
    "mp_max_bits": ([], _u32),
    "mp_version": ([], ctypes.c_char_p),
    "mp_convert": ([_vp, _i, _vp, _i, _sz, _u32, _vp], _i),
    "mp_mul": ([_vp, _vp, _vp, _sz, _u32, _i, _i, _vp], _i),
    "mp_sqr": ([_vp, _vp, _sz, _u32, _i, _i, _vp], _i),
    "mont_ctx_init": ([ctypes.POINTER(_vp), _vp, _sz, _u32, _i, ctypes.POINTER(_sz), _vp], _i),
    "mont_ctx_free": ([_vp], _i),
    "mont_ctx_info": ([_vp, ctypes.POINTER(_sz), ctypes.POINTER(_u32), ctypes.POINTER(_i)], _i),
    "mont_ctx_export": ([_vp, _i, _vp, _vp], _i),
    "mont_mul": ([_vp, _vp, _vp, _vp, _i, _i, _vp], _i),
    "mont_sqr": ([_vp, _vp, _vp, _i, _i, _vp], _i),
    "modexp_workspace_bytes": ([_sz, _u32, _u32], _sz),
    "modexp_consttime": ([_vp, _vp, _vp, _u32, _vp, _u32, _i, _i, _vp, _sz, _vp], _i),
    "mp_bench_imad": ([_i, _i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _vp], _i),
    "modexp_consttime_noalloc": ([_vp, _vp, _vp, _u32, _vp, _u32, _i, _i, _vp], _i),
    "mp_noalloc_scratch_bytes": ([], ctypes.c_size_t),
    "modexp_timing_probe": ([_vp, _vp, _vp, _vp, _u32, _vp, _u32, _i, _vp, _sz, _vp], _i),
    "mp_shape_candidates": ([_u32, ctypes.POINTER(_i), ctypes.POINTER(_i), _i], _i),
    "mp_tune_set": ([_u32, _i, _i, _u32, _u32], _i),
    "mp_tune_get": ([_u32, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_u32), ctypes.POINTER(_u32)], _i),
    "mp_tune_set_mont_karatsuba": ([_u32, _u32], _i),
    "mp_tune_get_mont_karatsuba": ([_u32, ctypes.POINTER(_u32)], _i),
    "mp_shape_residency": ([_u32, _i, _i, _i, _i, ctypes.POINTER(_i)], _i),
    "mp_tune_set_table": ([_u32, _i], _i),
    "mp_debug_bounds": ([ctypes.POINTER(ctypes.c_ulonglong)], _i),
    "mp_debug_bounds_selftest": ([_vp], _i),
    "mp_tune_get_table": ([_u32, ctypes.POINTER(_i)], _i),
    "mp_table_residency": ([_u32, _u32, ctypes.POINTER(_i)], _i),
    "modexp_mixed_workspace_bytes": ([_vp, _i], _sz),
    "modexp_consttime_mixed": ([_vp, _i, _i, _vp, _sz, _vp], _i),
    "modexp_table_bytes": ([_vp, _u32], _sz),
    "modexp_table_build": ([_vp, _sz, _vp, _vp, _u32, _i, _vp], _i),
    "modexp_fixed_base": ([_vp, _vp, _vp, _u32, _sz, _vp, _vp, _u32, _i, _vp], _i),
}
for _name, (_args, _res) in _SIG.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_SIG)


class MpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {_lib.mp_strerror(status).decode()} ({status})")


def _check(st: int, where: str):
    if st != 0:
        raise MpError(st, where)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if t.element_size() != 4:
        raise ValueError("expected a 32-bit integer tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def words(bits: int) -> int:
    return (int(bits) + 31) // 32


def max_bits() -> int:
    return int(_lib.mp_max_bits())


def version() -> str:
    return _lib.mp_version().decode()


def array_words(layout: int, batch: int, w: int) -> int:
    """Words of an array of `batch` values of `w` words in `layout`."""
    return ((w + 3) // 4) * 4 * batch if layout == LAYOUT_INTERLEAVED else w * batch


def mp_convert(dst: torch.Tensor, dst_layout: int, src: torch.Tensor, src_layout: int, batch: int, w: int):
    _check(_lib.mp_convert(_ptr(dst), dst_layout, _ptr(src), src_layout, batch, w, _stream()), "mp_convert")
    return dst


def mp_mul(c, a, b, batch: int, bits: int, layout: int = LAYOUT_INSTANCE_MAJOR, algo: int = ALGO_AUTO):
    _check(_lib.mp_mul(_ptr(c), _ptr(a), _ptr(b), batch, bits, layout, algo, _stream()), "mp_mul")
    return c


def mp_sqr(c, a, batch: int, bits: int, layout: int = LAYOUT_INSTANCE_MAJOR, algo: int = ALGO_AUTO):
    _check(_lib.mp_sqr(_ptr(c), _ptr(a), batch, bits, layout, algo, _stream()), "mp_sqr")
    return c


class MontCtx:
    """Owns a mont_ctx (device copies of N, N', R mod N, R^2 mod N)."""

    def __init__(self, N: torch.Tensor, batch: int, bits: int, layout: int = LAYOUT_INSTANCE_MAJOR):
        h = ctypes.c_void_p()
        bad = ctypes.c_size_t(0)
        st = _lib.mont_ctx_init(ctypes.byref(h), _ptr(N), batch, bits, layout, ctypes.byref(bad), _stream())
        if st == -3:
            err = MpError(st, "mont_ctx_init")
            err.bad_index = int(bad.value)
            raise err
        _check(st, "mont_ctx_init")
        self.handle = h
        self.batch, self.bits, self.layout = batch, bits, layout
        self.n = words(bits)

    def export(self, which: int) -> torch.Tensor:
        out = torch.zeros(array_words(self.layout, self.batch, self.n), dtype=torch.int32, device="cuda")
        _check(_lib.mont_ctx_export(self.handle, which, _ptr(out), _stream()), "mont_ctx_export")
        return out

    def free(self):
        if self.handle:
            _check(_lib.mont_ctx_free(self.handle), "mont_ctx_free")
            self.handle = None

    def __del__(self):
        try:
            if getattr(self, "handle", None):
                _lib.mont_ctx_free(self.handle)
        except Exception:
            pass


def mont_ctx_init(N, batch: int, bits: int, layout: int = LAYOUT_INSTANCE_MAJOR) -> MontCtx:
    return MontCtx(N, batch, bits, layout)


def mont_mul(c, a, b, ctx: MontCtx, red: int = RED_TRUNCATED, algo: int = ALGO_AUTO):
    _check(_lib.mont_mul(_ptr(c), _ptr(a), _ptr(b), ctx.handle, red, algo, _stream()), "mont_mul")
    return c


def mont_sqr(c, a, ctx: MontCtx, red: int = RED_TRUNCATED, algo: int = ALGO_AUTO):
    _check(_lib.mont_sqr(_ptr(c), _ptr(a), ctx.handle, red, algo, _stream()), "mont_sqr")
    return c


def modexp_workspace_bytes(batch: int, bits: int, window: int) -> int:
    return int(_lib.modexp_workspace_bytes(batch, bits, window))


def modexp_consttime(y, base, exp, exp_bits: int, ctx: MontCtx, window: int = 0,
                     red: int = RED_TRUNCATED, algo: int = ALGO_AUTO, workspace: torch.Tensor | None = None):
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(_lib.modexp_consttime(_ptr(y), _ptr(base), _ptr(exp), exp_bits, ctx.handle, window, red, algo,
                                 _ptr(workspace), ws_bytes, _stream()), "modexp_consttime")
    return y


NOALLOC_SCRATCH_BYTES = int(_lib.mp_noalloc_scratch_bytes())   # the library's static array


class _Job(ctypes.Structure):
    _fields_ = [("y", ctypes.c_void_p), ("base", ctypes.c_void_p), ("exp", ctypes.c_void_p),
                ("exp_bits", ctypes.c_uint32), ("window", ctypes.c_uint32), ("ctx", ctypes.c_void_p),
                ("index", ctypes.c_void_p), ("tables", ctypes.c_void_p), ("nreq", ctypes.c_size_t)]


def _jobs(jobs):
    """jobs: sequence of (y, base, exp, exp_bits, ctx, window) for exponentiations of a
    context's own bases, or (y, base, exp, exp_bits, ctx, window, index, tables, nreq) for
    requests routed to context instances: fixed-base on resident tables (base None, tables
    given) or with their own bases (tables None) -> ctypes array."""
    arr = (_Job * len(jobs))()
    for i, job in enumerate(jobs):
        y, base, exp, exp_bits, ctx, window = job[:6]
        if len(job) > 6:
            index, tables, nreq = job[6:9]
            arr[i] = _Job(_ptr(y), _ptr(base), _ptr(exp), exp_bits, window, ctx.handle, _ptr(index), _ptr(tables),
                          nreq)
        else:
            arr[i] = _Job(_ptr(y), _ptr(base), _ptr(exp), exp_bits, window, ctx.handle, None, None, 0)
    return arr


def modexp_table_bytes(ctx: MontCtx, window: int) -> int:
    return int(_lib.modexp_table_bytes(ctx.handle, window))


def modexp_table_build(tables: torch.Tensor, base, ctx: MontCtx, window: int, red: int = RED_TRUNCATED):
    _check(_lib.modexp_table_build(_ptr(tables), tables.numel() * tables.element_size(), _ptr(base), ctx.handle,
                                   window, red, _stream()), "modexp_table_build")
    return tables


def modexp_fixed_base(y, index, exp, exp_bits: int, nreq: int, ctx: MontCtx, tables: torch.Tensor, window: int,
                      red: int = RED_TRUNCATED):
    _check(_lib.modexp_fixed_base(_ptr(y), _ptr(index), _ptr(exp), exp_bits, nreq, ctx.handle, _ptr(tables),
                                  window, red, _stream()), "modexp_fixed_base")
    return y


def modexp_mixed_workspace_bytes(jobs) -> int:
    arr = _jobs(jobs)
    return int(_lib.modexp_mixed_workspace_bytes(arr, len(jobs)))


def modexp_consttime_mixed(jobs, red: int = RED_TRUNCATED, workspace: torch.Tensor | None = None):
    """One call over several jobs of any sizes (see _jobs): each job runs its size class's kernel,
    the jobs forked onto parallel streams costliest first and joined back to the current stream."""
    arr = _jobs(jobs)
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(_lib.modexp_consttime_mixed(arr, len(jobs), red, _ptr(workspace), ws_bytes, _stream()),
           "modexp_consttime_mixed")


def mixed_workspace(jobs) -> torch.Tensor:
    """A 256-byte-aligned device buffer large enough for these jobs."""
    nbytes = modexp_mixed_workspace_bytes(jobs)
    if nbytes == 0:
        raise MpError(-1, "modexp_mixed_workspace_bytes")
    return torch.empty((nbytes + 255) // 256 * 64, dtype=torch.int32, device="cuda")


def shape_candidates(bits: int):
    G = (ctypes.c_int * 8)()
    M = (ctypes.c_int * 8)()
    k = _lib.mp_shape_candidates(bits, G, M, 8)
    if k < 0:
        raise MpError(k, "mp_shape_candidates")
    return [(G[i], M[i]) for i in range(min(k, 8))]


def tune_set(bits: int, G: int = 0, M: int = 0, window: int = 0, karatsuba_from_bits: int = 0):
    _check(_lib.mp_tune_set(bits, G, M, window, karatsuba_from_bits), "mp_tune_set")


def tune_get(bits: int):
    G, M, w, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(_lib.mp_tune_get(bits, ctypes.byref(G), ctypes.byref(M), ctypes.byref(w), ctypes.byref(k)),
           "mp_tune_get")
    return {"G": G.value, "M": M.value, "window": w.value, "karatsuba_from_bits": k.value}


def tune_set_mont_karatsuba(bits: int, karatsuba_from_bits: int):
    _check(_lib.mp_tune_set_mont_karatsuba(bits, karatsuba_from_bits), "mp_tune_set_mont_karatsuba")


def tune_get_mont_karatsuba(bits: int) -> int:
    k = ctypes.c_uint32()
    _check(_lib.mp_tune_get_mont_karatsuba(bits, ctypes.byref(k)), "mp_tune_get_mont_karatsuba")
    return k.value


def debug_bounds() -> int:
    """Debug builds: the first recorded bounds violation (0: none), then cleared; synchronises the
    device. Release builds raise MpError (MP_ERR_UNIMPLEMENTED)."""
    v = ctypes.c_ulonglong()
    _check(_lib.mp_debug_bounds(ctypes.byref(v)), "mp_debug_bounds")
    return v.value


def debug_bounds_selftest():
    """Debug builds: record one self-test violation (kind 6) without any memory access."""
    _check(_lib.mp_debug_bounds_selftest(_stream()), "mp_debug_bounds_selftest")


def tune_set_table(bits: int, placement: int):
    """Window-table placement of modexp_consttime for the class of `bits` (TABLE_GLOBAL or
    TABLE_SHARED; see mp_tune_set_table)."""
    _check(_lib.mp_tune_set_table(bits, placement), "mp_tune_set_table")


def tune_get_table(bits: int) -> int:
    p = _i()
    _check(_lib.mp_tune_get_table(bits, ctypes.byref(p)), "mp_tune_get_table")
    return p.value


def table_residency(bits: int, window: int) -> int:
    """Instances per SM of the exponentiation with shared-memory window tables (0: they do not fit)."""
    r = _i()
    _check(_lib.mp_table_residency(bits, window, ctypes.byref(r)), "mp_table_residency")
    return r.value


def shape_residency(bits: int, G: int = 0, M: int = 0, red: int = RED_TRUNCATED, algo: int = ALGO_AUTO) -> int:
    """Instances of the exponentiation kernel resident on one SM (see mp_shape_residency)."""
    r = ctypes.c_int()
    _check(_lib.mp_shape_residency(bits, G, M, red, algo, ctypes.byref(r)), "mp_shape_residency")
    return r.value


def modexp_timing_probe(cycles: torch.Tensor, y, base, exp, exp_bits: int, ctx: MontCtx, window: int,
                        red: int, workspace: torch.Tensor):
    """modexp_consttime that also writes each instance's SM clock cycles into `cycles` (an int32
    tensor of 2 x batch words, read through .view(torch.int64))."""
    _check(_lib.modexp_timing_probe(_ptr(cycles), _ptr(y), _ptr(base), _ptr(exp), exp_bits, ctx.handle, window, red,
                                    _ptr(workspace), workspace.numel() * workspace.element_size(), _stream()),
           "modexp_timing_probe")
    return cycles


def modexp_consttime_noalloc(y, base, exp, exp_bits: int, ctx: MontCtx, window: int = 0,
                             red: int = RED_TRUNCATED, algo: int = ALGO_AUTO):
    """modexp_consttime with its window tables in the library's fixed device array
    (no allocation; at most NOALLOC_SCRATCH_BYTES of tables; concurrent calls race)."""
    _check(_lib.modexp_consttime_noalloc(_ptr(y), _ptr(base), _ptr(exp), exp_bits, ctx.handle, window, red,
                                         algo, _stream()), "modexp_consttime_noalloc")
    return y


def bench_imad(mode: int, iters: int = 2000):
    """(rate per SM per clock, implied SM MHz) of the integer microbenchmark `mode`."""
    r, mhz = ctypes.c_double(0), ctypes.c_double(0)
    _check(_lib.mp_bench_imad(mode, iters, ctypes.byref(r), ctypes.byref(mhz), _stream()), "mp_bench_imad")
    return r.value, mhz.value


# --------------------------------------------------------------------------- host helpers

def to_device(x, device="cuda") -> torch.Tensor:
    """numpy uint32 array -> int32 CUDA tensor with the same bits."""
    import numpy as np
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int32)).to(device)


def to_host(t: torch.Tensor):
    import numpy as np
    return t.detach().cpu().numpy().view(np.uint32)


def interleave(x):
    """[batch, w] instance-major numpy -> flat interleaved numpy (host-side reshaping only)."""
    import numpy as np
    B, w = x.shape
    c = (w + 3) // 4
    pad = np.zeros((B, c * 4), np.uint32)
    pad[:, :w] = x
    return np.ascontiguousarray(pad.reshape(B, c, 4).transpose(1, 0, 2)).reshape(-1)


def deinterleave(flat, batch: int, w: int):
    import numpy as np
    c = (w + 3) // 4
    return np.ascontiguousarray(np.asarray(flat, np.uint32).reshape(c, batch, 4).transpose(1, 0, 2)
                                ).reshape(batch, c * 4)[:, :w]
