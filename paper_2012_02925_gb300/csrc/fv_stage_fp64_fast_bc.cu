// Fused stage kernel instantiated for the binary64 form: default scheme compiled in, boundary-face
// flux overwrites.
#include "fv_stage.cuh"

int fv_launch_stage_fp64_fast_bc(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s) {
  return fv_dispatch_launch<double, true, false, true>(a, l, s);
}
int fv_stage_occupancy_fp64_fast_bc(const FvLaunch& l, size_t* smem) {
  return fv_dispatch_occupancy<double, true, false, true>(l, smem);
}
