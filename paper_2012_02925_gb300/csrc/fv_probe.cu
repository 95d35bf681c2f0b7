// Arithmetic throughput probe of the GPU the library runs on: the measured
// peaks the fused stage kernel's arithmetic roofline is graded against.
//
// Each probe kernel runs CHAINS independent dependency chains per thread of
// one operation (enough independent work per warp to keep its pipe busy),
// on a grid of 8 CTAs of 256 threads per SM; the rate is operations executed
// / device time (CUDA events, best of three launches after a warm-up).  The
// chains' results feed a store that never happens at run time, so nothing is
// optimised away.  binary64 operations are the hardware's (DFMA, DADD, DMUL)
// and the compiler's IEEE reciprocal and square root, and the face code's
// own reciprocal (fv_rcp64); the double-float operations are those of
// fv_arith.cuh.
#include <cuda_runtime.h>

#include "../../include/fvgb.h"
#include "fv_arith.cuh"

namespace {

constexpr int CHAINS = 8;
constexpr int THREADS = 256;

enum ProbeOp {
  P_DFMA, P_DADD, P_DMUL, P_DRCP, P_DSQRT, P_FFMA, P_DF_ADD, P_DF_MUL, P_DF_DIV, P_DF_SQRT, P_DF_ABS, P_DRCPN,
  P_DSQRTN
};

template <int OP>
__global__ void __launch_bounds__(THREADS) probe_fp64(int iters, double seed, double* sink) {
  double x[CHAINS];
  const double t = seed + 1e-7 * (threadIdx.x + blockIdx.x);
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = t + 0.25 * c + 1.5;
  const double a = 0.9999999, b = 1e-7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
      if (OP == P_DFMA) x[c] = fma(x[c], a, b);
      if (OP == P_DADD) x[c] = x[c] + b;
      if (OP == P_DMUL) x[c] = x[c] * a;
      if (OP == P_DRCP) x[c] = 1.0 / x[c];
      if (OP == P_DSQRT) x[c] = sqrt(x[c]);
      if (OP == P_DRCPN) x[c] = fv_rcp64(x[c]);
      if (OP == P_DSQRTN) x[c] = fv_sqrt64(x[c]);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  if (s == 1.2345e-300) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(THREADS) probe_ffma(int iters, float seed, double* sink) {
  float x[CHAINS];
  const float t = seed + 1e-7f * (threadIdx.x + blockIdx.x);
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = t + 0.25f * c + 1.5f;
  const float a = 0.9999f, b = 1e-4f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = __fmaf_rn(x[c], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  if (s == 1.2345e-30f) sink[threadIdx.x] = s;
}

template <int OP>
__global__ void __launch_bounds__(THREADS) probe_df64(int iters, float seed, double* sink) {
  df64 x[CHAINS];
  const float t = seed + 1e-5f * (threadIdx.x + blockIdx.x);
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = mk(t + 0.25f * c + 1.5f, 1e-9f);
  const df64 a = mk(0.9999999f, 3e-15f), b = mk(1e-7f, 1e-16f), one = mk(1.0f, 0.0f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
      if (OP == P_DF_ADD) x[c] = x[c] + b;
      if (OP == P_DF_MUL) x[c] = x[c] * a;
      if (OP == P_DF_DIV) x[c] = one / x[c];
      if (OP == P_DF_SQRT) x[c] = df_sqrt(x[c]);
      if (OP == P_DF_ABS) x[c] = -df_abs(x[c]);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c].hi + x[c].lo;
  if (s == 1.2345e-30f) sink[threadIdx.x] = s;
}

// best of three timed launches after one warm-up: operations per second
template <class F>
double time_rate(F launch, double ops, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, int* err) {
  launch();
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) { *err = 1; return 0.0; }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms > 0.0f && ms < best) best = ms;
  }
  if (cudaGetLastError() != cudaSuccess) *err = 1;
  return ops / (best * 1e-3);
}

}  // namespace

extern "C" int fv_probe_alu_rates(double* out_host, int n_out, void* stream) {
  if (!out_host || n_out < FV_PROBE_NRATES) return FV_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FV_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FV_ERR_CUDA;
  const int grid = 8 * nsm;
  double* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * THREADS) != cudaSuccess) return FV_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const double threads = (double)grid * THREADS * CHAINS;
  int err = 0;
  // iteration counts: a few milliseconds per launch at GB300's rates
  const int it_d = 512, it_slow = 64, it_f = 16384, it_df = 1024, it_dfs = 256;
#define FV_PROBE_D(OP, IT) \
  time_rate([&] { probe_fp64<OP><<<grid, THREADS, 0, s>>>(IT, 0.5, sink); }, threads * (IT), s, e0, e1, &err)
#define FV_PROBE_DF(OP, IT) \
  time_rate([&] { probe_df64<OP><<<grid, THREADS, 0, s>>>(IT, 0.5f, sink); }, threads * (IT), s, e0, e1, &err)
  out_host[0] = FV_PROBE_D(P_DFMA, it_d);
  out_host[1] = FV_PROBE_D(P_DADD, it_d);
  out_host[2] = FV_PROBE_D(P_DMUL, it_d);
  out_host[3] = FV_PROBE_D(P_DRCP, it_slow);
  out_host[4] = FV_PROBE_D(P_DSQRT, it_slow);
  out_host[5] = time_rate([&] { probe_ffma<<<grid, THREADS, 0, s>>>(it_f, 0.5f, sink); }, threads * it_f, s, e0, e1,
                          &err);
  out_host[6] = FV_PROBE_DF(P_DF_ADD, it_df);
  out_host[7] = FV_PROBE_DF(P_DF_MUL, it_df);
  out_host[8] = FV_PROBE_DF(P_DF_DIV, it_dfs);
  out_host[9] = FV_PROBE_DF(P_DF_SQRT, it_dfs);
  out_host[10] = FV_PROBE_DF(P_DF_ABS, it_df);
  out_host[11] = FV_PROBE_D(P_DRCPN, it_slow);
  out_host[12] = FV_PROBE_D(P_DSQRTN, it_slow);
#undef FV_PROBE_D
#undef FV_PROBE_DF
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  return err ? FV_ERR_CUDA : FV_OK;
}

// ---------------------------------------------------------------------------
// binary64 reciprocal and square-root checks: the face code's reciprocal
// and square root next to the compiler's IEEE 1.0 / x and sqrt(x), for a
// test on the host
// ---------------------------------------------------------------------------
namespace {
template <bool SQRT>
__global__ void arith_check_kernel(const double* __restrict__ x, long long n, double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    out[2 * i] = SQRT ? fv_sqrt64(x[i]) : fv_rcp64(x[i]);
    out[2 * i + 1] = SQRT ? sqrt(x[i]) : 1.0 / x[i];
  }
}

int arith_check(const void* kernel, const double* x_dev, int64_t n, double* out_dev, void* stream) {
  if (!x_dev || !out_dev || n <= 0) return FV_ERR_INVALID_ARG;
  const long long blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
  long long nn = n;
  void* args[] = {&x_dev, &nn, &out_dev};
  if (cudaLaunchKernel(kernel, dim3((unsigned)blocks), dim3(256), args, 0, (cudaStream_t)stream) != cudaSuccess)
    return FV_ERR_CUDA;
  return FV_OK;
}
}  // namespace

extern "C" int fv_check_rcp64(const double* x_dev, int64_t n, double* out_dev, void* stream) {
  return arith_check((const void*)arith_check_kernel<false>, x_dev, n, out_dev, stream);
}

extern "C" int fv_check_sqrt64(const double* x_dev, int64_t n, double* out_dev, void* stream) {
  return arith_check((const void*)arith_check_kernel<true>, x_dev, n, out_dev, stream);
}
