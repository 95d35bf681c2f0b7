// Fused stage kernel instantiated for the binary64 form: generic scheme switches, boundary-face
// flux overwrites.
#include "fv_stage.cuh"

int fv_launch_stage_fp64_bc(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s) {
  return fv_dispatch_launch<double, false, false, true>(a, l, s);
}
int fv_stage_occupancy_fp64_bc(const FvLaunch& l, size_t* smem) {
  return fv_dispatch_occupancy<double, false, false, true>(l, smem);
}
