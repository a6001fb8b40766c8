// hzn_adj_general.cu -- reverse substep kernels for a general 3+1 metric.
#include "hzn_adjoint.cuh"

namespace hzn {
namespace adj {

template void adj_launch_cell<false>(bool, int, int, cudaStream_t, const KParams&, const AdjShape&,
                                    const double*, const double*, const AdjBufs&);
template void adj_launch_face<false>(bool, dim3, int, cudaStream_t, const KParams&, const AdjShape&,
                                    const double*, const double*, const AdjBufs&);

}  // namespace adj
}  // namespace hzn
