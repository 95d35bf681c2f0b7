// Fused stage kernel instantiated for the binary64 form: generic scheme switches, laminar viscous
// pairs of the separate viscous kernel, boundary-face flux overwrites.
#include "fv_stage.cuh"

int fv_launch_stage_fp64_visc_bc(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s) {
  return fv_dispatch_launch<double, false, true, true>(a, l, s);
}
int fv_stage_occupancy_fp64_visc_bc(const FvLaunch& l, size_t* smem) {
  return fv_dispatch_occupancy<double, false, true, true>(l, smem);
}
