// Debug builds (compiled with -DMPG_DEBUG_BOUNDS): bounds checks on the kernels' shared-memory
// block accesses (lds / sts: inside the block's shared memory, 16-byte aligned for vector
// accesses), on the words of the global arrays they read and write (gload / gstore: inside the
// array of `batch` instances in its layout) and on the window-table entries of the
// exponentiations. A failed check records its first occurrence in this translation unit's debug
// word (kind in the top byte, the offending offset below it) and the access is skipped (a load
// gives zeros); nothing traps, so a faulty index shows up as a recorded violation and wrong
// results, never as a device fault. Release builds compile none of it.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mpg {

enum DbgKind : uint32_t { DBG_SMEM = 1, DBG_ALIGN = 2, DBG_LOAD = 3, DBG_STORE = 4, DBG_TABLE = 5, DBG_SELFTEST = 6 };

#ifdef MPG_DEBUG_BOUNDS
static __device__ unsigned long long g_mpg_dbg;   // one per translation unit (internal linkage)

__device__ __forceinline__ bool dbg_ok(bool ok, uint32_t kind, unsigned long long where) {
    if (!ok) atomicCAS(&g_mpg_dbg, 0ull, ((unsigned long long)kind << 56) | (where & ((1ull << 56) - 1)));
    return ok;
}

// the block's dynamic shared memory: every extern __shared__ array starts there (the kernels of
// this library use no static shared memory), and %dynamic_smem_size is its size at launch
extern __shared__ uint4 mpg_dbg_dyn_smem[];

// `bytes` bytes at p lie inside the block's dynamic shared memory (and are 16-byte aligned if
// `vec`)
__device__ __forceinline__ bool smem_ok(const void *p, int bytes, bool vec) {
    if (!__isShared(p)) return dbg_ok(false, DBG_SMEM, 0xffffffffull);
    const uint32_t off = (uint32_t)__cvta_generic_to_shared(p);
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(mpg_dbg_dyn_smem);
    uint32_t size;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(size));
    if (!dbg_ok(off >= base && off - base + (uint32_t)bytes <= size, DBG_SMEM, off - base)) return false;
    return dbg_ok(!vec || (off & 15u) == 0u, DBG_ALIGN, off - base);
}

// host: this unit's debug word, then cleared (~0 if it could not be read)
static unsigned long long dbg_take() {
    unsigned long long v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_mpg_dbg, sizeof v) != cudaSuccess) return ~0ull;
    if (cudaMemcpyToSymbol(g_mpg_dbg, &z, sizeof z) != cudaSuccess) return ~0ull;
    return v;
}
#define MPG_DBG_TAKE (&dbg_take)
#else
__device__ __forceinline__ bool dbg_ok(bool, uint32_t, unsigned long long) { return true; }
__device__ __forceinline__ bool smem_ok(const void *, int, bool) { return true; }
#define MPG_DBG_TAKE nullptr
#endif

}  // namespace mpg
