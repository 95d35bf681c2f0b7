// Fused stage kernel instantiated for the binary32-flux form: default scheme compiled in, no
// boundary-face overwrites.
#include "fv_stage.cuh"

int fv_launch_stage_fp32_fast(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s) {
  return fv_dispatch_launch<float, true, false, false>(a, l, s);
}
int fv_stage_occupancy_fp32_fast(const FvLaunch& l, size_t* smem) {
  return fv_dispatch_occupancy<float, true, false, false>(l, smem);
}
