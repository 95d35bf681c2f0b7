// Fused stage kernel instantiated for the binary32-flux form: generic scheme switches, laminar
// viscous terms fused into the face loop, no boundary-face overwrites.
#include "fv_stage.cuh"

int fv_launch_stage_fp32_visc(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s) {
  return fv_dispatch_launch<float, false, true, false>(a, l, s);
}
int fv_stage_occupancy_fp32_visc(const FvLaunch& l, size_t* smem) {
  return fv_dispatch_occupancy<float, false, true, false>(l, smem);
}
