// Fused stage kernel instantiated for the binary64 form with the laminar viscous pairs of the separate viscous kernel, generic scheme switches.
#include "fv_stage.cuh"

int fv_launch_stage_fp64_visc(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s) {
  return fv_dispatch_launch<double, false, true>(a, l, s);
}
int fv_stage_occupancy_fp64_visc(const FvLaunch& l, size_t* smem) { return fv_dispatch_occupancy<double, false, true>(l, smem); }
