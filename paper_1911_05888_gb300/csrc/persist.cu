// Persistent coarse cycle: the part of Algorithm 1 below a chosen level (its
// colour steps, residuals, restrictions, coarse visits, bottom solve and
// prolongations) run as ONE cooperative launch that walks a precomputed
// program of phases, with a grid barrier between consecutive phases instead
// of a kernel boundary.
//
// On the coarse levels a colour step has few elements (64 x 64 and below: at
// most 1024), so a launch per step is bound by launch and dependency latency
// rather than by bytes: the whole coarse part of one V(3,3) cycle of the
// 256 x 256 workload is about 110 such steps.  Here each phase is a grid-
// stride loop of the same per-element / per-coarse-element bodies the
// standalone kernels run (element_core.cuh), so a phase gives the same bits as
// the launch it replaces.
//
// The grid barrier spins with a bound: a CTA that waits longer than `limit`
// clock ticks sets the context's error word and returns, every other CTA sees
// the word at its next barrier and returns too, and the host reports
// STK_ERR_TIMEOUT.  The launch is cooperative, so all CTAs are co-resident and
// a correct program never reaches the bound.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "element_core.cuh"
#include "stk_internal.h"

namespace stk {

namespace {

// Bounded sense-counting grid barrier.  count: arrivals at the current
// barrier; gen: barriers completed.  Returns false when the error word is set
// (by this CTA after `limit` ticks, or by another CTA).
__device__ __forceinline__ bool grid_barrier(GridBarrierWords* gb, int* err, long long limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* vgen = &gb->gen;
    const unsigned int my = *vgen;
    __threadfence();
    const unsigned int nblocks = gridDim.x;
    if (atomicAdd(&gb->count, 1u) == nblocks - 1) {
      atomicExch(&gb->count, 0u);
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == my) {
        if (*(volatile int*)err != 0) {
          ok = 0;
          break;
        }
        if (clock64() - t0 > limit) {
          atomicExch(err, kErrBarrierTimeout);
          ok = 0;
          break;
        }
        __nanosleep(40);
      }
    }
    __threadfence();
    s_ok = ok && *(volatile int*)err == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename TS, typename TX, int S>
__global__ void __launch_bounds__(kWideNT) coarse_cycle_kernel(const __grid_constant__ Pattern pat,
                                                               const WideGeom wg,
                                                               const CyclePhase* __restrict__ phases, int nphase,
                                                               GridBarrierWords* gb, int* err, long long limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int d = pat.d, s = pat.s, nb = pat.nb;
  for (int ph = 0; ph < nphase; ++ph) {
    const CyclePhase P = phases[ph];
    if (P.op == PHASE_GS || P.op == PHASE_RESID) {
      const int mode = P.op == PHASE_GS ? MODE_GS : MODE_RESID;
      for (int pos = P.pos0 + (int)blockIdx.x; pos < P.pos0 + (int)P.n; pos += gridDim.x)
        wide_element<TS, TX, S>(pat, wg, mode, pos, P.perm, P.nbr, (const TS*)P.cpl, (const TS*)P.mat, P.tsc,
                                P.rsc, (const TX*)P.b, (TX*)P.x, (TX*)P.r, smem_raw);
    } else if (P.op == PHASE_RESTRICT) {
      // r_c = I^T r, and the coarse iterate starts from zero (Algorithm 1)
      for (int64_t C = blockIdx.x; C < P.n; C += gridDim.x) {
        restrict_coarse<TX>(d, s, nb, P.dims[0], P.dims[1], P.dims[2], P.dims[3], C, (const TX*)P.tr,
                            (const TX*)P.in, (TX*)P.out, reinterpret_cast<TX*>(smem_raw));
        for (int i = threadIdx.x; i < nb; i += blockDim.x) ((TX*)P.xz)[C * nb + i] = (TX)0;
      }
    } else if (P.op == PHASE_PROLONG) {
      for (int64_t C = blockIdx.x; C < P.n; C += gridDim.x)
        prolong_coarse<TX>(d, s, nb, P.dims[0], P.dims[1], P.dims[2], P.dims[3], C, (const TX*)P.tr,
                           (const TX*)P.in, (TX*)P.out, reinterpret_cast<TX*>(smem_raw));
    } else if (P.op == PHASE_BOTTOM) {
      // x = A_c^+ b, one warp per row, FP64 accumulation (as bottom_kernel)
      const int lane = threadIdx.x & 31, warps = blockDim.x / 32;
      const double* pinv = (const double*)P.tr;
      const TX* bb = (const TX*)P.in;
      TX* xx = (TX*)P.out;
      for (int64_t row = (int64_t)blockIdx.x * warps + threadIdx.x / 32; row < P.n;
           row += (int64_t)gridDim.x * warps) {
        double acc = 0.0;
        for (int64_t j = lane; j < P.n; j += 32) acc += pinv[row * P.n + j] * (double)bb[j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) xx[row] = (TX)acc;
      }
    }
    if (ph + 1 < nphase && !grid_barrier(gb, err, limit)) return;
  }
}

// Barrier self-test: every CTA passes `rounds` barriers; CTA `absent` (when
// >= 0) returns at once and never arrives, so the others must give up after
// `limit` ticks with the error word set.
__global__ void barrier_selftest_kernel(GridBarrierWords* gb, int* err, long long limit, int rounds, int absent,
                                        unsigned int* passed) {
  if ((int)blockIdx.x == absent) return;
  for (int k = 0; k < rounds; ++k) {
    if (!grid_barrier(gb, err, limit)) return;
    if (threadIdx.x == 0) atomicAdd(passed, 1u);
  }
}

template <typename TS, typename TX, int S>
cudaError_t launch_coarse_s(const Pattern& pat, const CyclePhase* phases, int nphase, GridBarrierWords* gb, int* err,
                            long long limit, int grid, cudaStream_t st) {
  const WideGeom wg = wide_geometry<TS>(pat);
  using TA = typename StorageTraits<TS>::Acc;
  size_t smem = kMaxOffsets * sizeof(int) + wg.words * sizeof(TA);
  const size_t tr = (size_t)(1 << pat.d) * pat.nb * sizeof(TX);   // transfer staging
  if (tr > smem) smem = tr;
  if (smem > 226 * 1024) return cudaErrorInvalidValue;
  auto kern = coarse_cycle_kernel<TS, TX, S>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0, dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWideNT, smem)) != cudaSuccess) return e;
  if (per_sm < 1 || grid < 1 || grid > per_sm * sms) return cudaErrorInvalidValue;   // must be co-resident
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kWideNT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, pat, wg, phases, nphase, gb, err, limit);
}

template <typename TS, typename TX>
cudaError_t launch_coarse_t(const Pattern& pat, const CyclePhase* phases, int nphase, GridBarrierWords* gb, int* err,
                            long long limit, int grid, cudaStream_t st) {
#define STK_COARSE_CASE(SV) \
  case SV: return launch_coarse_s<TS, TX, SV>(pat, phases, nphase, gb, err, limit, grid, st);
  switch (pat.s) {
    STK_COARSE_CASE(4)
    STK_COARSE_CASE(8)
    STK_COARSE_CASE(9)
    STK_COARSE_CASE(16)
    STK_COARSE_CASE(25)
    STK_COARSE_CASE(27)
    default: return cudaErrorInvalidValue;
  }
#undef STK_COARSE_CASE
}

}  // namespace

cudaError_t launch_coarse_cycle(const Pattern& pat, int storage, const CyclePhase* phases, int nphase,
                                GridBarrierWords* gb, int* err, long long limit, int grid, cudaStream_t st) {
  if (nphase < 1) return cudaSuccess;
  switch (storage) {
    case 0: return launch_coarse_t<double, double>(pat, phases, nphase, gb, err, limit, grid, st);
    case 1: return launch_coarse_t<float, float>(pat, phases, nphase, gb, err, limit, grid, st);
    case 2: return launch_coarse_t<__nv_bfloat16, float>(pat, phases, nphase, gb, err, limit, grid, st);
    case 3: return launch_coarse_t<__half, float>(pat, phases, nphase, gb, err, limit, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_barrier_selftest(GridBarrierWords* gb, int* err, long long limit, int rounds, int absent, int grid,
                                    unsigned int* passed, cudaStream_t st) {
  int per_sm = 0, sms = 0, dev = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, barrier_selftest_kernel, 64, 0)) != cudaSuccess)
    return e;
  if (grid < 1 || grid > per_sm * sms) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(64);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, barrier_selftest_kernel, gb, err, limit, rounds, absent, passed);
}

}  // namespace stk
