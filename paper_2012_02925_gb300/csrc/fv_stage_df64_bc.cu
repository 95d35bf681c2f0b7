// Fused stage kernel instantiated for the double-float form: generic scheme switches, boundary-face
// flux overwrites.
#include "fv_stage.cuh"

int fv_launch_stage_df64_bc(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s) {
  return fv_dispatch_launch<df64, false, false, true>(a, l, s);
}
int fv_stage_occupancy_df64_bc(const FvLaunch& l, size_t* smem) {
  return fv_dispatch_occupancy<df64, false, false, true>(l, smem);
}
