// hzn_internal.h -- structures shared by the host API and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hzn {

// Device-resident scalars: the time-step clock and the run statistics.
struct DevScalars {
  unsigned long long vmax_bits;  // max speed / dx of the newest state (bits of a positive double)
  unsigned long long fails;      // recovery failures since hz_set_primitives
  int maxit;                     // largest Newton iteration count
  unsigned int metric_general;   // set by the metric scan: nonzero shift or off-diagonal gamma
  double dt;                     // dt of the step in flight
  double t;                      // simulated time
  long long steps;
};

struct KParams {
  int nx, ny, nz;
  int bcx, bcy, bcz;
  int pitch;             // x pitch of the interior arrays
  long long plane;       // pitch * ny
  long long fs;          // field stride of the interior arrays
  int mpitch, mny;       // metric x pitch, metric y extent
  long long mplane;      // mpitch * mny
  long long ms;          // metric field stride
  int gx, gy, gz;        // metric ghost widths
  double idx, idy, idz;  // 1 / dx
  double gamma, gfac, ch, kappa;
  double rho_floor, rho_atm, p_floor, p_atm;
  int c2p_maxit;
  double c2p_tol;
  double c2p_step_tol;   // Newton stops once a step is below this (0.01 sqrt(c2p_tol), relative)
  int c2p_1d;            // 1: the 1D recovery scheme (Newton in z, v^2 eliminated)
  int zlen;              // cells of z per block (the chunked grid of the mixed and pair kernels)
  int nsm;               // SMs of the device the context was created on
  int dev;               // that device's ordinal
  // Geometry tables of a metric with zero shift and diagonal gamma (filled by hz_set_metric,
  // used by the DIAG kernels), in the metric's padded layout (field stride ms):
  //   geo_c  centre geometry, GEO_C fields (both precisions; FP64 values): the GEO_N fields
  //          of Geom, then sum over active axes of alpha sqrt(gamma^dd) / dx_d (the CFL rate of a
  //          state at rest per unit signal speed);
  //   geo_f  face geometry of axis d at geo_f + d GEO_F ms, the face i - 1/2 of cell (i, j, k)
  //          at the cell's metric offset: the GEO_N fields of the centre table, then
  //          alpha sqrt(gamma^dd) (the cleaning speed per unit c_h) (FP64 path only);
  //   geo_s  differences g(+1) - g(-1) of g_tt, g_xx, g_yy, g_zz along axis d at
  //          geo_s + d GEO_S ms (FP64 path only).
  const double* geo_c;
  const double* geo_f;
  const double* geo_s;
  // FP32 copies of the constants of the FP32 face arithmetic (filled by set_float_consts), so
  // that the kernels load them instead of converting the doubles per face
  float f_gamma, f_gfac, f_ch, f_ch2, f_idx, f_idy, f_idz, f_kappa, f_rho_floor, f_p_atm;
};

// Fill the FP32 copies of KParams' constants from the doubles (host side, once per context).
inline void set_float_consts(KParams& kp) {
  kp.f_gamma = (float)kp.gamma;
  kp.f_gfac = (float)kp.gfac;
  kp.f_ch = (float)kp.ch;
  kp.f_ch2 = (float)(kp.ch * kp.ch);
  kp.f_idx = (float)kp.idx;
  kp.f_idy = (float)kp.idy;
  kp.f_idz = (float)kp.idz;
  kp.f_kappa = (float)kp.kappa;
  kp.f_rho_floor = (float)kp.rho_floor;
  kp.f_p_atm = (float)kp.p_atm;
}

constexpr int GEO_N = 10;  // alpha, 1/alpha, gamma_xx, _yy, _zz, gamma^xx, ^yy, ^zz, sqrt(gamma), sqrt(-g)
constexpr int GEO_C = GEO_N + 1;  // centre table: GEO_N fields and sum_d alpha sqrt(gamma^dd) / dx_d
constexpr int GEO_F = GEO_N + 1;  // face tables: GEO_N fields and alpha sqrt(gamma^dd)
constexpr int GEO_S = 4;   // g_tt, g_xx, g_yy, g_zz

// One substep: Uout = a0 U0 + ak (Uk + dt L(Pin)); Pout = primitives of Uout.
struct StageArgs {
  const void* Pin;       // primitive state (double, or float in the mixed path)
  void* Pout;
  const double* U0;
  const double* Uk;
  double* Uout;
  double a0, ak;
  int last;              // 1 on the last substep: accumulate the CFL maximum
};

#ifdef __CUDACC__
// The CUDA runtime error behind an HZ_ERR_CUDA: records e (when it is an error) as the calling
// host thread's last one (hz_last_cuda_error) and returns HZ_OK or HZ_ERR_CUDA.
int record_cuda_error(cudaError_t e);
#endif

// Which instantiation to launch.
struct Variant {
  int dims;    // 1, 2 or 3 active axes (x, then y, then z)
  int clean;   // divergence cleaning
  int diag;    // zero shift and diagonal gamma everywhere
  int mixed;   // FP32 storage of P and metric, FP32 faces/sources
  int recon;   // 0 MC, 1 PPM
  int pair;    // FP64 state with double-word (f32x2) faces, fluxes and sources
};

// Launchers, one per (precision, dims) translation unit; dispatch in hzn_dispatch.cu.
void launch_substep(const Variant& v, const KParams& kp, const StageArgs& sa, const void* M,
                    DevScalars* sc, int zchunks, cudaStream_t st);
void launch_prim2cons(const Variant& v, const KParams& kp, const void* P, const void* M, double* U,
                      cudaStream_t st);
void launch_max_speed(const Variant& v, const KParams& kp, const void* P, const void* M,
                      DevScalars* sc, cudaStream_t st);
void launch_geo_tables(const Variant& v, const KParams& kp, const void* M, double* geo_c,
                       double* geo_f, double* geo_s, cudaStream_t st);

// Tile shape of the substep kernel per dimensionality.
inline void tile_of(int dims, int* tx, int* ty) {
  *tx = 32;
  *ty = dims == 1 ? 1 : 4;
}

}  // namespace hzn
