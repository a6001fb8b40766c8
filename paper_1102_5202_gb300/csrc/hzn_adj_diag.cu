// hzn_adj_diag.cu -- reverse substep kernels for zero shift and a diagonal spatial metric (geometry from the tables).
#include "hzn_adjoint.cuh"

namespace hzn {
namespace adj {

template void adj_launch_cell<true>(bool, int, int, cudaStream_t, const KParams&, const AdjShape&,
                                    const double*, const double*, const AdjBufs&);
template void adj_launch_face<true>(bool, dim3, int, cudaStream_t, const KParams&, const AdjShape&,
                                    const double*, const double*, const AdjBufs&);

}  // namespace adj
}  // namespace hzn
