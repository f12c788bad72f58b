// Allocation-free residual + norm entry point (see stk_residual_norm_static in
// include/stokes_mg.h).
//
// Its only scratch memory -- the per-chunk partial sums of ||r||^2 -- lives in
// a file-scope __device__ array instead of memory the library allocates, so a
// call never reaches cudaMalloc or any allocating routine.  Host code cannot
// use the array's name as a device address (in host code it names a host-side
// shadow); the device address is fetched once per device with
// cudaGetSymbolAddress while that device is current.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "stk_internal.h"
#include "../../include/stokes_mg.h"

namespace {

constexpr int kChunk = 2048;                      // entries summed by one partial (256 x 8)
constexpr int kStaticPartials = 16384;            // 128 KB of doubles
constexpr int64_t kMaxUnknowns = (int64_t)kChunk * kStaticPartials;   // 33,554,432
constexpr int kMaxDevices = 64;

// Scratch of every call on a device: partial sums, one per chunk.  Each call
// writes every slot it later reads, so nothing needs clearing between calls;
// calls that run concurrently on one device share (and race on) this array.
static __device__ __align__(256) double g_static_partials[kStaticPartials];

std::mutex g_lock;
double* g_partials_addr[kMaxDevices] = {nullptr};

__global__ void chunk_sumsq_kernel(int64_t n, const double* __restrict__ x, double* __restrict__ part) {
  __shared__ double sh[256];
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  double acc = 0.0;
  for (int i = threadIdx.x; i < kChunk; i += 256) {
    const int64_t j = base + i;
    if (j < n) acc += x[j] * x[j];
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void partials_total_kernel(int nparts, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 256) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

// Device address of g_static_partials on `device` (which must be current),
// fetched on the first call on that device and kept for the life of the
// process: a cudaDeviceReset (or unloading the library) invalidates it.
cudaError_t partials_address(int device, double** out) {
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_partials_addr[device]) {
    double* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&p, g_static_partials);
    if (e != cudaSuccess) return e;
    g_partials_addr[device] = p;
  }
  *out = g_partials_addr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" int stk_residual_norm_static(stk_ctx* c, const double* x, const double* b, double* r,
                                        double* norm2_dev, void* stream) {
  if (!c) return STK_ERR_INVALID_ARG;
  if (!c->ready) {
    c->err = "call stk_setup first";
    return STK_ERR_NOT_SETUP;
  }
  if (!x || !b || !r || !norm2_dev) {
    c->err = "null vector";
    return STK_ERR_INVALID_ARG;
  }
  if (c->device < 0 || c->device >= kMaxDevices) {
    c->err = "device index beyond the static-scratch table";
    return STK_ERR_INVALID_ARG;
  }
  const int64_t n = (int64_t)c->host[0].ne * c->nb;
  const int64_t nparts = (n + kChunk - 1) / kChunk;
  if (n > kMaxUnknowns) {
    c->err = "stk_residual_norm_static: problem has more than 33554432 unknowns on level 0, "
             "the capacity of its fixed scratch; use stk_residual";
    return STK_ERR_INVALID_ARG;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    c->err = "cudaGetDevice failed";
    return STK_ERR_CUDA;
  }
  if (prev != c->device && cudaSetDevice(c->device) != cudaSuccess) {
    c->err = "cudaSetDevice failed";
    return STK_ERR_CUDA;
  }
  int rc = STK_OK;
  double* part = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = partials_address(c->device, &part);
  if (e == cudaSuccess) {
    // The same launch as stk_residual: the FP64 residual on the kernel
    // variant the context's tuning picks for level 0 (none of them allocates).
    const stk::DevLevel& D = c->dev[0];
    e = stk::run_element(*c, 0, STK_FP64, stk::MODE_RESID, 0, D.ne, D.dia[0], b, (void*)x, r, st);
  }
  if (e == cudaSuccess) {
    chunk_sumsq_kernel<<<(unsigned)nparts, 256, 0, st>>>(n, r, part);
    partials_total_kernel<<<1, 256, 0, st>>>((int)nparts, part, norm2_dev);
    e = cudaGetLastError();
    c->launches += 3;
  }
  if (e != cudaSuccess) {
    c->err = cudaGetErrorString(e);
    rc = STK_ERR_CUDA;
  }
  if (prev != c->device) cudaSetDevice(prev);
  return rc;
}
