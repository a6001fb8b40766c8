// Instantiations of the FP64 kernels with PPM reconstruction for 2-D grids (a unit of
// its own so that the build runs the heavy instantiations in parallel).
#include "hzn_kernels.cuh"

namespace hzn {

void launch_substep_k64p_2d(const Variant& v, const KParams& kp, const StageArgs& sa, const void* M,
                            DevScalars* sc, int zchunks, cudaStream_t st) {
  launch_substep_t<true, false, false, 1>(v, kp, sa, M, sc, zchunks, st);
}

}  // namespace hzn
