// The persistent mixed-size kernel with the classical reduction (Alg. 5).
#include "mp_mixed.cuh"
namespace mpg {
cudaError_t launch_mixed_red1(const MixArgs &P, cudaStream_t st) { return launch_mixed<1>(P, st); }
}  // namespace mpg
