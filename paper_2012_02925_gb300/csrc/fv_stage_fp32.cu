// Fused stage kernel instantiated for the binary32-flux form: generic scheme switches, no
// boundary-face overwrites.
#include "fv_stage.cuh"

int fv_launch_stage_fp32(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s) {
  return fv_dispatch_launch<float, false, false, false>(a, l, s);
}
int fv_stage_occupancy_fp32(const FvLaunch& l, size_t* smem) {
  return fv_dispatch_occupancy<float, false, false, false>(l, smem);
}
