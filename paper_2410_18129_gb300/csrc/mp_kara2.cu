// Two-level Karatsuba products: 4096-bit class (quarters of 8 threads x 4 words) and
// 4608-bit class, which holds 4108 and 4154 bits (quarters of 4 threads x 9 words).
#include "mp_kara.cuh"
namespace mpg {
cudaError_t kara2_128(const KArgs &A, cudaStream_t st) { return launch_kara2<Shape<8, 4>, 128>(A, st); }
cudaError_t kara2_144(const KArgs &A, cudaStream_t st) { return launch_kara2<Shape<4, 9>, 64>(A, st); }
#ifdef MPG_DEBUG_BOUNDS
unsigned long long dbg_take_kara2() { return dbg_take(); }
#else
unsigned long long dbg_take_kara2() { return 0; }
#endif
}  // namespace mpg
