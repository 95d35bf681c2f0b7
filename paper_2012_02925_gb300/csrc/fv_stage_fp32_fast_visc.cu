// Fused stage kernel instantiated for the binary32-flux form with the laminar viscous terms, default scheme compiled in.
#include "fv_stage.cuh"

int fv_launch_stage_fp32_fast_visc(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s) {
  return fv_dispatch_launch<float, true, true>(a, l, s);
}
int fv_stage_occupancy_fp32_fast_visc(const FvLaunch& l, size_t* smem) { return fv_dispatch_occupancy<float, true, true>(l, smem); }
