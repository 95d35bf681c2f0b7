// Fused stage kernel instantiated for the double-float form: generic scheme switches, laminar
// viscous pairs of the separate viscous kernel, no boundary-face overwrites.
#include "fv_stage.cuh"

int fv_launch_stage_df64_visc(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s) {
  return fv_dispatch_launch<df64, false, true, false>(a, l, s);
}
int fv_stage_occupancy_df64_visc(const FvLaunch& l, size_t* smem) {
  return fv_dispatch_occupancy<df64, false, true, false>(l, smem);
}
