// The persistent mixed-size kernel with the word-serial CIOS reduction (Alg. 4).
#include "mp_mixed.cuh"
namespace mpg {
cudaError_t launch_mixed_red2(const MixArgs &P, cudaStream_t st) { return launch_mixed<2>(P, st); }
}  // namespace mpg
