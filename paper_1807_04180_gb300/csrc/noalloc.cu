// Allocation-free norms of complex128 vectors (ddm_norms_noalloc).
//
// The two-pass reduction behind ddm_residual's norms keeps its per-block partial sums in
// device scratch that the context allocates.  Some callers cannot allocate device memory
// at the point where they need a norm: code that runs under a fixed memory budget, inside
// a caching allocator it must not re-enter, or in a section where cudaMalloc would stall
// other streams by synchronising the device.  For them this variant keeps its scratch in
// a file-scope device array instead: NA_BLOCKS x NA_MAX_VEC partial sums plus NA_MAX_VEC
// totals (about 39 KB), held by every GPU that loads the library until the process exits.
#include <math.h>

#include <mutex>
#include <string>

#include "ddm_internal.cuh"

namespace ddm {
void set_global_error(const std::string& msg);
}

namespace {

constexpr int NA_BLOCKS = 304;    // reduction blocks (2 per SM of a GB300)
constexpr int NA_MAX_VEC = 16;    // largest number of vectors per call
constexpr int NA_MAX_DEV = 64;    // device ordinals with a cached scratch address

// partial sums [NA_BLOCKS][NA_MAX_VEC], then the NA_MAX_VEC totals
static __device__ __align__(256) double g_na_scratch[NA_BLOCKS * NA_MAX_VEC + NA_MAX_VEC];

std::mutex g_na_mu;
double* g_na_addr[NA_MAX_DEV] = {nullptr};

__device__ __forceinline__ double na_block_sum(double v, double* sh) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;
}

// part[blk * NA_MAX_VEC + v] = sum of |x_v[i]|^2 over this block's grid-stride share
__global__ void k_na_partial(const ddm::z64* x, long long n, int nvec, double* part) {
  __shared__ double sh[32];
  for (int v = 0; v < nvec; ++v) {
    double s = 0;
    const ddm::z64* xv = x + (long long)v * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
      s += xv[i].x * xv[i].x + xv[i].y * xv[i].y;
    double t = na_block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x * NA_MAX_VEC + v] = t;
  }
}

// out[v] = sqrt(sum over blocks of part[. * NA_MAX_VEC + v]) (one block per vector)
__global__ void k_na_total(const double* part, double* out) {
  __shared__ double sh[32];
  const int v = blockIdx.x;
  double s = 0;
  for (int b = threadIdx.x; b < NA_BLOCKS; b += blockDim.x) s += part[b * NA_MAX_VEC + v];
  double t = na_block_sum(s, sh);
  if (threadIdx.x == 0) out[v] = sqrt(t);
}

ddm_status na_fail(ddm_status st, const std::string& msg) {
  ddm::set_global_error(msg);
  return st;
}

}  // namespace

extern "C" ddm_status ddm_norms_noalloc(const void* x_dev, int64_t n, int nvec, void* stream, double* norms_dev) {
  if (!x_dev || !norms_dev) return na_fail(DDM_E_INVAL, "ddm_norms_noalloc: null pointer");
  if (n < 1) return na_fail(DDM_E_INVAL, "ddm_norms_noalloc: n must be >= 1");
  if (nvec < 1 || nvec > NA_MAX_VEC)
    return na_fail(DDM_E_INVAL, "ddm_norms_noalloc: nvec must be in [1, 16] (static scratch holds 16 vectors)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(DDM_E_CUDA, std::string("ddm_norms_noalloc: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= NA_MAX_DEV) return na_fail(DDM_E_INVAL, "ddm_norms_noalloc: device ordinal beyond 63");
  double* scratch = nullptr;
  {
    // once per device, with that device current: the host-side name of g_na_scratch is only a
    // stand-in, so kernels get the device address from cudaGetSymbolAddress.  The address is
    // kept for the life of the process; after cudaDeviceReset (or any teardown of the device's
    // primary context) it is stale, and the call must not be used again in that process.
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_na_scratch);
      if (e != cudaSuccess || !p)
        return na_fail(DDM_E_CUDA, std::string("ddm_norms_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_na_addr[dev] = (double*)p;
    }
    scratch = g_na_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  // clear a launch error left by unrelated earlier work, so that the check below reports only
  // this call's launches (a sticky error from a faulted context is not cleared and fails here)
  (void)cudaGetLastError();
  k_na_partial<<<NA_BLOCKS, 256, 0, st>>>((const ddm::z64*)x_dev, (long long)n, nvec, scratch);
  k_na_total<<<nvec, 256, 0, st>>>(scratch, norms_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(DDM_E_CUDA, std::string("ddm_norms_noalloc: ") + cudaGetErrorString(e));
  return DDM_OK;
}
