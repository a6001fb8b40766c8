// Dispatch of the kernel launchers on dimensionality, precision and reconstruction.
#include "hzn_kernels.cuh"

namespace hzn {

#define HZN_DECLARE(P, D)                                                                          \
  void launch_substep_k##P##_##D##d(const Variant&, const KParams&, const StageArgs&, const void*, \
                                    DevScalars*, int, cudaStream_t);                               \
  void launch_max_speed_k##P##_##D##d(const Variant&, const KParams&, const void*, const void*,    \
                                      DevScalars*, cudaStream_t);
HZN_DECLARE(64, 1)
HZN_DECLARE(64, 2)
HZN_DECLARE(64, 3)
HZN_DECLARE(32, 1)
HZN_DECLARE(32, 2)
HZN_DECLARE(32, 3)
#undef HZN_DECLARE
#define HZN_DECLARE_PPM(P, D)                                                                      \
  void launch_substep_k##P##p_##D##d(const Variant&, const KParams&, const StageArgs&, const void*, \
                                     DevScalars*, int, cudaStream_t);
HZN_DECLARE_PPM(64, 1)
HZN_DECLARE_PPM(64, 2)
HZN_DECLARE_PPM(64, 3)
HZN_DECLARE_PPM(32, 1)
HZN_DECLARE_PPM(32, 2)
HZN_DECLARE_PPM(32, 3)
#undef HZN_DECLARE_PPM
#define HZN_DECLARE_PAIR(D)                                                                        \
  void launch_substep_k64x_##D##d(const Variant&, const KParams&, const StageArgs&, const void*,  \
                                  DevScalars*, int, cudaStream_t);
HZN_DECLARE_PAIR(1)
HZN_DECLARE_PAIR(2)
HZN_DECLARE_PAIR(3)
#undef HZN_DECLARE_PAIR

void launch_substep(const Variant& v, const KParams& kp, const StageArgs& sa, const void* M,
                    DevScalars* sc, int zchunks, cudaStream_t st) {
  if (v.recon) {
    if (v.mixed) {
      if (v.dims == 1) launch_substep_k32p_1d(v, kp, sa, M, sc, zchunks, st);
      else if (v.dims == 2) launch_substep_k32p_2d(v, kp, sa, M, sc, zchunks, st);
      else launch_substep_k32p_3d(v, kp, sa, M, sc, zchunks, st);
    } else {
      if (v.dims == 1) launch_substep_k64p_1d(v, kp, sa, M, sc, zchunks, st);
      else if (v.dims == 2) launch_substep_k64p_2d(v, kp, sa, M, sc, zchunks, st);
      else launch_substep_k64p_3d(v, kp, sa, M, sc, zchunks, st);
    }
    return;
  }
  if (v.pair) {
    if (v.dims == 1) launch_substep_k64x_1d(v, kp, sa, M, sc, zchunks, st);
    else if (v.dims == 2) launch_substep_k64x_2d(v, kp, sa, M, sc, zchunks, st);
    else launch_substep_k64x_3d(v, kp, sa, M, sc, zchunks, st);
    return;
  }
  if (v.mixed) {
    if (v.dims == 1) launch_substep_k32_1d(v, kp, sa, M, sc, zchunks, st);
    else if (v.dims == 2) launch_substep_k32_2d(v, kp, sa, M, sc, zchunks, st);
    else launch_substep_k32_3d(v, kp, sa, M, sc, zchunks, st);
  } else {
    if (v.dims == 1) launch_substep_k64_1d(v, kp, sa, M, sc, zchunks, st);
    else if (v.dims == 2) launch_substep_k64_2d(v, kp, sa, M, sc, zchunks, st);
    else launch_substep_k64_3d(v, kp, sa, M, sc, zchunks, st);
  }
}

void launch_max_speed(const Variant& v, const KParams& kp, const void* P, const void* M,
                      DevScalars* sc, cudaStream_t st) {
  if (v.mixed) {
    if (v.dims == 1) launch_max_speed_k32_1d(v, kp, P, M, sc, st);
    else if (v.dims == 2) launch_max_speed_k32_2d(v, kp, P, M, sc, st);
    else launch_max_speed_k32_3d(v, kp, P, M, sc, st);
  } else {
    if (v.dims == 1) launch_max_speed_k64_1d(v, kp, P, M, sc, st);
    else if (v.dims == 2) launch_max_speed_k64_2d(v, kp, P, M, sc, st);
    else launch_max_speed_k64_3d(v, kp, P, M, sc, st);
  }
}

void launch_geo_tables(const Variant& v, const KParams& kp, const void* M, double* geo_c,
                       double* geo_f, double* geo_s, cudaStream_t st) {
  const long long n = (long long)(kp.nx + 1) * (kp.ny + kp.gy) * (kp.nz + kp.gz);
  const int nb = blocks_for(n, 256);
  if (v.mixed) k_geo_tables<float><<<nb, 256, 0, st>>>(kp, (const float*)M, geo_c, geo_f, geo_s, 0);
  else k_geo_tables<double><<<nb, 256, 0, st>>>(kp, (const double*)M, geo_c, geo_f, geo_s, 1);
}

void launch_prim2cons(const Variant& v, const KParams& kp, const void* P, const void* M, double* U,
                      cudaStream_t st) {
  if (v.mixed) launch_prim2cons_t<true>(v, kp, P, M, U, st);
  else launch_prim2cons_t<false>(v, kp, P, M, U, st);
}

}  // namespace hzn
