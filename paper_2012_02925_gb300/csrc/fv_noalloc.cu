// Residual-norm reduction that allocates nothing.
//
// fv_residual_norms() keeps its per-CTA partial sums in device memory that the
// handle allocates with cudaMalloc on first use.  Some callers cannot allow
// that: code running under a framework's caching allocator (where a
// cudaMalloc would synchronise the device or fragment the pool), embedded or
// real-time hosts that forbid allocation after start-up, and plugins that
// only ever receive memory from their host application.  fv_field_norms_noalloc() serves them: the caller passes the
// field and the output buffer, and the partial sums live in a fixed,
// file-scope device array that is part of the loaded library.
//
// That array (1024 slots x 5 variables x 3 values = 120 KiB) exists
// on every GPU that loads the library and stays allocated until the process
// exits.  All calls share it and it keeps the contents of the last call; each
// call writes every slot it later reads, so nothing has to be cleared, but two
// calls whose kernels overlap on the GPU (different streams, no ordering
// between them) race on it.
#include <mutex>

#include "../../include/fvgb.h"

namespace {

constexpr int kParts = FV_NOALLOC_MAX_N / FV_NOALLOC_CHUNK;   // partial-sum slots
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// [variable][sum | max | non-finite][slot]
static __device__ __align__(256) double g_norm_scratch[5 * 3 * kParts];

double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_norm_scratch on the current device.  In host code the
// symbol name is only a host-side stand-in, so the address must be queried
// once per device, with that device current.  The address is kept for the
// life of the process: a cudaDeviceReset() of a device unloads the module
// and invalidates it, so a process that resets a device must not call this
// entry point on that device afterwards.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FV_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return FV_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_norm_scratch) != cudaSuccess || !p) return FV_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return FV_OK;
}

// CTA p reduces elements [p*CHUNK, (p+1)*CHUNK) of each of the 5 planes.
__global__ void __launch_bounds__(kThreads) chunk_norms(const double* __restrict__ f, long long n,
                                                        double* __restrict__ scratch) {
  __shared__ double ssum[kThreads / 32], smax[kThreads / 32];
  __shared__ int sbad[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long lo = (long long)blockIdx.x * FV_NOALLOC_CHUNK;
  const long long hi = lo + FV_NOALLOC_CHUNK < n ? lo + FV_NOALLOC_CHUNK : n;
  for (int v = 0; v < 5; ++v) {
    const double* fv = f + (long long)v * n;
    double s = 0.0, m = 0.0;
    int bad = 0;
    for (long long x = lo + threadIdx.x; x < hi; x += kThreads) {
      const double y = fv[x];
      bad |= !isfinite(y);
      s += y * y;
      m = fmax(m, fabs(y));
    }
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_down_sync(0xffffffffu, s, o);
      m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
      bad |= __shfl_down_sync(0xffffffffu, bad, o);
    }
    if (lane == 0) { ssum[warp] = s; smax[warp] = m; sbad[warp] = bad; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double ts = 0.0, tm = 0.0;
      int tb = 0;
      for (int w = 0; w < kThreads / 32; ++w) { ts += ssum[w]; tm = fmax(tm, smax[w]); tb |= sbad[w]; }
      scratch[(v * 3 + 0) * kParts + blockIdx.x] = ts;
      scratch[(v * 3 + 1) * kParts + blockIdx.x] = tm;
      scratch[(v * 3 + 2) * kParts + blockIdx.x] = tb;
    }
    __syncthreads();
  }
}

__global__ void finish_norms(const double* __restrict__ scratch, int parts, long long n, double* __restrict__ out) {
  __shared__ double flag[5];
  const int v = threadIdx.x;
  if (v < 5) {
    double s = 0.0, m = 0.0, b = 0.0;
    for (int p = 0; p < parts; ++p) {
      s += scratch[(v * 3 + 0) * kParts + p];
      m = fmax(m, scratch[(v * 3 + 1) * kParts + p]);
      b += scratch[(v * 3 + 2) * kParts + p];
    }
    out[v] = sqrt(s / (double)n);
    out[5 + v] = m;
    flag[v] = b != 0.0 ? 1.0 : 0.0;
  }
  __syncthreads();
  if (v == 0) out[10] = flag[0] + flag[1] + flag[2] + flag[3] + flag[4];
}

}  // namespace

extern "C" int fv_field_norms_noalloc(const double* field_dev, int64_t n, double* out_dev, void* stream) {
  if (!field_dev || !out_dev || n <= 0) return FV_ERR_INVALID_ARG;
  if (n > FV_NOALLOC_MAX_N) return FV_ERR_INVALID_ARG;
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != FV_OK) return rc;
  int parts = (int)((n + FV_NOALLOC_CHUNK - 1) / FV_NOALLOC_CHUNK);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // cudaLaunchKernel reports the status of this launch itself, so an error
  // another caller left in the thread's last-error slot is neither reported
  // here nor cleared
  long long nn = n;
  void* a1[] = {&field_dev, &nn, &scratch};
  if (cudaLaunchKernel((const void*)chunk_norms, dim3(parts), dim3(kThreads), a1, 0, s) != cudaSuccess)
    return FV_ERR_CUDA;
  void* a2[] = {&scratch, &parts, &nn, &out_dev};
  if (cudaLaunchKernel((const void*)finish_norms, dim3(1), dim3(32), a2, 0, s) != cudaSuccess) return FV_ERR_CUDA;
  return FV_OK;
}
