// Fused stage kernel instantiated for the double-float form: default scheme compiled in, no
// boundary-face overwrites.
#include "fv_stage.cuh"

int fv_launch_stage_df64_fast(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s) {
  return fv_dispatch_launch<df64, true, false, false>(a, l, s);
}
int fv_stage_occupancy_df64_fast(const FvLaunch& l, size_t* smem) {
  return fv_dispatch_occupancy<df64, true, false, false>(l, smem);
}
