// hzn_adj.h -- host-visible shapes and launchers of the reverse (adjoint) substep kernels.
//
// The kernels themselves (hzn_adjoint.cuh) are instantiated once per metric class in
// hzn_adj_diag.cu (zero shift, diagonal spatial metric: geometry from the precomputed tables)
// and hzn_adj_general.cu (general 3+1 metric); hzn_adjoint.cu drives them.
#pragma once

#include <cuda_runtime.h>

#include "hzn_internal.h"

namespace hzn {
namespace adj {

// Shapes of the adjoint arrays.  Cell arrays use the forward layout (kp.pitch, kp.plane,
// kp.fs); face arrays hold faces i - 1/2 for i = 0 .. n_D along D, one more cell per axis.
struct AdjShape {
  int fpitch;
  long long fplane, ffs;
  double dt;
  double a, b;     // stage coefficients of the substep whose implicit-function step runs
  int stage;       // 0, 1, 2 for that substep; 3: final (adjoint of the initial primitives)
  int gather;      // 1: gather lam_P from the faces of the later substep; 0: read lam_P
};

struct AdjBufs {
  double* lamP;    // adjoint of the primitive state at the current substep boundary
  double* lamU;    // adjoint of the conserved state there
  double* lamA;    // accumulated adjoint of the step's starting conserved state U0
  double* lamL;    // b dt mu of the substep being reversed (adjoint of L)
  double* fL[3];   // per axis: adjoint of the left reconstructed state, 9 fields
  double* fR[3];   // per axis: adjoint of the right reconstructed state
  double* out;     // final: adjoint of the initial primitives (padded layout)
};

template <bool DIAG>
void adj_launch_cell(bool clean, int blocks, int threads, cudaStream_t st, const KParams& kp,
                     const AdjShape& sh, const double* Pb, const double* M, const AdjBufs& bufs);
template <bool DIAG>
void adj_launch_face(bool clean, dim3 grid, int threads, cudaStream_t st, const KParams& kp,
                     const AdjShape& sh, const double* P, const double* M, const AdjBufs& bufs);

}  // namespace adj
}  // namespace hzn
