// Instantiations of the FP64 kernels for 1-D grids (compiled as a unit of its own so
// that the build runs the heavy instantiations in parallel).
#include "hzn_kernels.cuh"

namespace hzn {

void launch_substep_k64_1d(const Variant& v, const KParams& kp, const StageArgs& sa, const void* M,
                        DevScalars* sc, int zchunks, cudaStream_t st) {
  launch_substep_t<false, false, false, 0>(v, kp, sa, M, sc, zchunks, st);
}

void launch_max_speed_k64_1d(const Variant& v, const KParams& kp, const void* P, const void* M,
                          DevScalars* sc, cudaStream_t st) {
  launch_max_speed_t<false, false, false>(v, kp, P, M, sc, st);
}

}  // namespace hzn
