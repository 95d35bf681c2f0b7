// Fused stage kernel instantiated for the binary32-flux form: default scheme compiled in, laminar
// viscous terms fused into the face loop, boundary-face flux overwrites.
#include "fv_stage.cuh"

int fv_launch_stage_fp32_fast_visc_bc(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s) {
  return fv_dispatch_launch<float, true, true, true>(a, l, s);
}
int fv_stage_occupancy_fp32_fast_visc_bc(const FvLaunch& l, size_t* smem) {
  return fv_dispatch_occupancy<float, true, true, true>(l, smem);
}
