// Fused stage kernel instantiated for the binary64 form: default scheme compiled in, laminar
// viscous pairs of the separate viscous kernel, boundary-face flux overwrites.
#include "fv_stage.cuh"

int fv_launch_stage_fp64_fast_visc_bc(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s) {
  return fv_dispatch_launch<double, true, true, true>(a, l, s);
}
int fv_stage_occupancy_fp64_fast_visc_bc(const FvLaunch& l, size_t* smem) {
  return fv_dispatch_occupancy<double, true, true, true>(l, smem);
}
