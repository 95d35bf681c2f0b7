// Residual monitor: per-variable RMS and maximum of the residual that RK
// stage 1 computes anyway (R(Q^(0)), the residual of the state a step starts
// from), the convergence history of Sections 8.1-8.3, without a separate
// residual evaluation.  The fused stage kernel stores R in its accumulator's
// storage (binary64 for the binary64 form, (hi, lo) binary32 pairs for the
// others); these kernels reduce it in the same arithmetic - double-float
// squares and sums run on the binary32 units, which GB300 gives 64 times the
// binary64 rate.  Fixed partition and fixed reduction order: deterministic.
#include "fv_arith.cuh"
#include "fv_internal.h"

namespace {

constexpr int MON_THREADS = 256;

__device__ __forceinline__ double mon_ld(const double* r, long long i) { return r[i]; }
__device__ __forceinline__ df64 mon_ld(const float2* r, long long i) {
  const float2 v = r[i];
  return mk(v.x, v.y);
}
__device__ __forceinline__ bool mon_finite(double y) { return isfinite(y); }
__device__ __forceinline__ bool mon_finite(df64 y) { return isfinite(y.hi) && isfinite(y.lo); }
__device__ __forceinline__ double mon_shfl(double y, int o) { return __shfl_down_sync(0xffffffffu, y, o); }
__device__ __forceinline__ df64 mon_shfl(df64 y, int o) {
  return mk(__shfl_down_sync(0xffffffffu, y.hi, o), __shfl_down_sync(0xffffffffu, y.lo, o));
}

// per-CTA partial sums of R^2, maxima of |R| and non-finite flags of each
// variable: partials[(v * 3 + {0, 1, 2}) * gridDim.x + CTA].  One pass over
// the cells with the five variables' loads independent of each other (a
// pass per variable kept one dependent load chain per thread in flight)
template <class ST, class A>
__global__ void __launch_bounds__(MON_THREADS) monitor_partial_kernel(const ST* __restrict__ r, long long n,
                                                                      double* __restrict__ partials) {
  using S = Sc<A>;
  __shared__ A ssum[5][MON_THREADS / 32], smax[5][MON_THREADS / 32];
  __shared__ int sbad[MON_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  A s[5], m[5];
  int bad = 0;
#pragma unroll
  for (int v = 0; v < 5; ++v) { s[v] = S::c(0.0); m[v] = S::c(0.0); }
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n;
       x += (long long)gridDim.x * blockDim.x) {
    A y[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) y[v] = mon_ld(r + v * n, x);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      if (!mon_finite(y[v])) bad = 1;
      s[v] = s[v] + y[v] * y[v];
      const A ay = S::abs(y[v]);
      if (S::lt(m[v], ay)) m[v] = ay;
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    for (int o = 16; o > 0; o >>= 1) {
      s[v] = s[v] + mon_shfl(s[v], o);
      const A mo = mon_shfl(m[v], o);
      if (S::lt(m[v], mo)) m[v] = mo;
    }
    if (lane == 0) { ssum[v][warp] = s[v]; smax[v][warp] = m[v]; }
  }
  for (int o = 16; o > 0; o >>= 1) bad |= __shfl_down_sync(0xffffffffu, bad, o);
  if (lane == 0) sbad[warp] = bad;
  __syncthreads();
  if (threadIdx.x < 5) {
    const int v = threadIdx.x;
    A ts = S::c(0.0), tm = S::c(0.0);
    int tb = 0;
    for (int w = 0; w < MON_THREADS / 32; ++w) {
      ts = ts + ssum[v][w];
      if (S::lt(tm, smax[v][w])) tm = smax[v][w];
      tb |= sbad[w];
    }
    partials[(v * 3 + 0) * gridDim.x + blockIdx.x] = S::to_d(ts);
    partials[(v * 3 + 1) * gridDim.x + blockIdx.x] = S::to_d(tm);
    partials[(v * 3 + 2) * gridDim.x + blockIdx.x] = tb;
  }
}

// one warp per variable: out[v] = sqrt(sum / n), out[5 + v] = max,
// out[10 + v] = count of CTAs that saw a non-finite value
__global__ void monitor_final_kernel(const double* __restrict__ partials, int nparts, long long n, double* out) {
  const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (v >= 5) return;
  double s = 0.0, m = 0.0, b = 0.0;
  for (int p = lane; p < nparts; p += 32) {
    s += partials[(v * 3 + 0) * nparts + p];
    m = fmax(m, partials[(v * 3 + 1) * nparts + p]);
    b += partials[(v * 3 + 2) * nparts + p];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    out[v] = sqrt(s / (double)n);
    out[5 + v] = m;
    out[10 + v] = b;
  }
}

}  // namespace

int fv_monitor_reduce(const void* rmon, int binary64, long long ncell, double* partials, int nparts, double* out,
                      cudaStream_t s) {
  if (binary64)
    monitor_partial_kernel<double, double><<<nparts, MON_THREADS, 0, s>>>(static_cast<const double*>(rmon), ncell,
                                                                         partials);
  else
    monitor_partial_kernel<float2, df64><<<nparts, MON_THREADS, 0, s>>>(static_cast<const float2*>(rmon), ncell,
                                                                       partials);
  monitor_final_kernel<<<1, 160, 0, s>>>(partials, nparts, ncell, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
