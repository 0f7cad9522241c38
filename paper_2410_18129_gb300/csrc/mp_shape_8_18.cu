// Kernels for groups of 8 threads x 18 words per thread (144 words, 4608 bits), 128 threads per
// block; one-level Karatsuba role-swapped over half products of 8 roles x 9 words. Measured at a
// batch of 65536 (M products/s, mul / sqr): lane-mapped schoolbook 305 / 458 against role-swapped
// 8 x 18 schoolbook 301 / 393 (128 registers with spills); Karatsuba role-swapped 300 / 448
// against lane-mapped 274 / 356.
#include "mp_swap_prod.cuh"
#ifdef MPG_LANE_ONLY
MPG_DEFINE_SHAPE_KARA(8, 18, 128, 9, 128)
#else
namespace mpg {
ShapeOps shape_ops_8_18() {
    ShapeOps o = ShapeImpl<Shape<8, 18>, 128>::ops();
    o.kara = &launch_kara_swap<SwapKara<8, 9>>;
    return o;
}
}  // namespace mpg
#endif
