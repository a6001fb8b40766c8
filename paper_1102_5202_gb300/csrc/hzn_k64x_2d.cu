// Instantiations of the double-word face kernels over the FP64 state for 2-D grids (MC
// reconstruction; a unit of its own so that the build runs the heavy instantiations in parallel).
#include "hzn_kernels.cuh"

namespace hzn {

void launch_substep_k64x_2d(const Variant& v, const KParams& kp, const StageArgs& sa, const void* M,
                           DevScalars* sc, int zchunks, cudaStream_t st) {
  launch_substep_t<true, false, false, 0, true>(v, kp, sa, M, sc, zchunks, st);
}

}  // namespace hzn
