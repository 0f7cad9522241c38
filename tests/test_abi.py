"""The C ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/mpgpu.h declares. No compute calls (no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpgpu.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    return __graft_entry__._load_build_script().build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("mp_mul", "mp_sqr", "mont_ctx_init", "mont_mul", "mont_sqr", "modexp_consttime",
                 "mont_ctx_free", "mp_strerror", "mp_convert"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_host_only_calls_work(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.mp_strerror.restype = ctypes.c_char_p
    lib.mp_strerror.argtypes = [ctypes.c_int]
    assert lib.mp_strerror(0) == b"ok"
    assert b"even" in lib.mp_strerror(-3)
    lib.mp_max_bits.restype = ctypes.c_uint32
    assert lib.mp_max_bits() >= 4154
    lib.modexp_workspace_bytes.restype = ctypes.c_size_t
    lib.modexp_workspace_bytes.argtypes = [ctypes.c_size_t, ctypes.c_uint32, ctypes.c_uint32]
    assert lib.modexp_workspace_bytes(65536, 2048, 5) == 32 * 64 * 4 * 65536
    assert lib.modexp_workspace_bytes(1, 2048, 9) == 0


def test_argument_errors_are_host_side(lib_path):
    """Invalid arguments are rejected before any CUDA call (safe without a GPU)."""
    lib = ctypes.CDLL(lib_path)
    vp = ctypes.c_void_p
    lib.mp_mul.argtypes = [vp, vp, vp, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, vp]
    fake = vp(16)
    assert lib.mp_mul(None, fake, fake, 4, 1024, 0, 0, None) == -1           # null
    assert lib.mp_mul(fake, fake, fake, 0, 1024, 0, 0, None) == -1           # empty batch
    assert lib.mp_mul(fake, fake, fake, 4, 0, 0, 0, None) == -2              # zero bits
    assert lib.mp_mul(fake, fake, fake, 4, 1 << 20, 0, 0, None) == -2        # too large
    assert lib.mp_mul(fake, fake, fake, 4, 1024, 7, 0, None) == -1           # bad layout
    assert lib.mp_mul(fake, vp(18), fake, 4, 1024, 1, 0, None) == -4         # misaligned interleaved
    lib.mont_ctx_init.argtypes = [ctypes.POINTER(vp), vp, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_size_t), vp]
    h = vp()
    assert lib.mont_ctx_init(ctypes.byref(h), fake, 4, 1, 0, None, None) == -2
    assert lib.mont_ctx_init(None, fake, 4, 1024, 0, None, None) == -1


def test_noalloc_scratch_size_matches_the_header(lib_path):
    """The static array's size as built equals the header's constant and the binding's."""
    lib = ctypes.CDLL(lib_path)
    lib.mp_noalloc_scratch_bytes.restype = ctypes.c_size_t
    m = re.search(r"#define\s+MPGPU_NOALLOC_SCRATCH_BYTES\s+\((\d+)u\s*<<\s*(\d+)\)", open(HEADER).read())
    assert m, "header constant not found"
    assert lib.mp_noalloc_scratch_bytes() == int(m.group(1)) << int(m.group(2))


def test_tuning_calls_are_host_side(lib_path):
    """The tuning setters and getters only touch the library's size-class table: their checks
    and round trips need no GPU (values are restored afterwards)."""
    lib = ctypes.CDLL(lib_path)
    u32, i = ctypes.c_uint32, ctypes.c_int
    lib.mp_tune_set_table.argtypes = [u32, i]
    lib.mp_tune_get_table.argtypes = [u32, ctypes.POINTER(i)]
    lib.mp_table_residency.argtypes = [u32, u32, ctypes.POINTER(i)]
    lib.mp_tune_set_mont_karatsuba.argtypes = [u32, u32]
    lib.mp_tune_get_mont_karatsuba.argtypes = [u32, ctypes.POINTER(u32)]
    p = i(-1)
    assert lib.mp_tune_get_table(2048, ctypes.byref(p)) == 0 and p.value == 0     # global by default
    assert lib.mp_tune_set_table(2048, 1) == 0
    assert lib.mp_tune_get_table(2000, ctypes.byref(p)) == 0 and p.value == 1     # the same size class
    assert lib.mp_tune_get_table(1024, ctypes.byref(p)) == 0 and p.value == 0     # another class
    assert lib.mp_tune_set_table(2048, 0) == 0
    assert lib.mp_tune_set_table(2048, 2) == -1                                  # no such placement
    assert lib.mp_tune_set_table(0, 0) == -2 and lib.mp_tune_set_table(1 << 20, 0) == -2
    assert lib.mp_tune_get_table(2048, None) == -1
    assert lib.mp_table_residency(2048, 0, ctypes.byref(p)) == -1                # window 0
    assert lib.mp_table_residency(2048, 7, ctypes.byref(p)) == -1                # window above 6
    assert lib.mp_table_residency(2048, 5, None) == -1
    k = u32(1)
    assert lib.mp_tune_get_mont_karatsuba(3072, ctypes.byref(k)) == 0 and k.value == 0
    assert lib.mp_tune_set_mont_karatsuba(3072, 3000) == 0
    assert lib.mp_tune_get_mont_karatsuba(3072, ctypes.byref(k)) == 0 and k.value == 3000
    assert lib.mp_tune_set_mont_karatsuba(3072, 0) == 0


def test_debug_build_compiles_and_exports(lib_path):
    """The bounds-checking variant (-DMPG_DEBUG_BOUNDS) cross-compiles here too and exports the same
    boundary, so its GPU test cannot fail on a build break alone."""
    import __graft_entry__
    dbg = __graft_entry__._load_build_script().build(debug=True)
    assert dbg != lib_path and os.path.exists(dbg)
    out = subprocess.run(["nm", "-D", "--defined-only", dbg], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    assert not [n for n in declared_functions() if n not in exported]
