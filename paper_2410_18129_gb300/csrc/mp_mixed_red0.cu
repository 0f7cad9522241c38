// The persistent mixed-size kernel with the truncated reduction (Alg. 6).
#include "mp_mixed.cuh"
namespace mpg {
cudaError_t launch_mixed_red0(const MixArgs &P, cudaStream_t st) { return launch_mixed<0>(P, st); }
}  // namespace mpg
