// Fused stage kernel instantiated for the binary32-flux form: default scheme compiled in,
// boundary-face flux overwrites.
#include "fv_stage.cuh"

int fv_launch_stage_fp32_fast_bc(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s) {
  return fv_dispatch_launch<float, true, false, true>(a, l, s);
}
int fv_stage_occupancy_fp32_fast_bc(const FvLaunch& l, size_t* smem) {
  return fv_dispatch_occupancy<float, true, false, true>(l, smem);
}
