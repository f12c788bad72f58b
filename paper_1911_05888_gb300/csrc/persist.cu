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

#include <algorithm>
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
  bool staged = false;   // this CTA's first element of the phase has its records in flight already
  for (int ph = 0; ph < nphase; ++ph) {
    const CyclePhase P = phases[ph];
    if (P.op == PHASE_GS || P.op == PHASE_RESID) {
      const int mode = P.op == PHASE_GS ? MODE_GS : MODE_RESID;
      for (int pos = P.pos0 + (int)blockIdx.x; pos < P.pos0 + (int)P.n; pos += gridDim.x) {
        wide_element<TS, TX, S>(pat, wg, mode, pos, P.perm, P.nbr, (const TS*)P.cpl, (const TS*)P.mat, P.tsc,
                                P.rsc, (const TX*)P.b, (TX*)P.x, (TX*)P.r, smem_raw, staged);
        staged = false;
      }
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
    staged = false;
    if (ph + 1 < nphase) {
      // records are never written: start the next phase's first element copy
      // now, so that it overlaps the barrier
      const CyclePhase& N = phases[ph + 1];
      if (wg.prefetch && (N.op == PHASE_GS || N.op == PHASE_RESID) && (int)blockIdx.x < (int)N.n) {
        __syncthreads();
        wide_stage<TS>(pat, wg, N.pos0 + (int)blockIdx.x, (const TS*)N.cpl, (const TS*)N.mat, smem_raw);
        staged = true;
      }
      if (!grid_barrier(gb, err, limit)) {
        if (staged) cp_async_wait_all();   // no copy may outlive the launch's shared memory
        return;
      }
    }
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
  size_t smem = wide_smem_bytes(wg);
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

// ---- batched outer iteration ----------------------------------------------------
// Every unit of a batch step is one warp's: an element (the warp-per-element
// body of the bandwidth kernel), a coarse element of a transfer, a bottom
// row, or a chunk of kBatchChunk vector entries.  Each warp owns a slice of
// the CTA's shared memory.
template <int S>
__device__ __forceinline__ void batch_element(const Pattern& pat, int op, const CyclePhase& P, int pos, void* wsm) {
  if (op == PHASE_RESID64) {
    const WarpGeom<double> wg = warp_geometry<double>(pat);
    warp_element<double, double, S>(pat, wg, MODE_RESID, pos, P.perm, P.nbr, (const double*)P.cpl,
                                    (const double*)P.mat, nullptr, nullptr, (const double*)P.b, (double*)P.x,
                                    (double*)P.r, wsm);
  } else {
    const WarpGeom<float> wg = warp_geometry<float>(pat);
    warp_element<float, float, S>(pat, wg, op == PHASE_GS ? MODE_GS : MODE_RESID, pos, P.perm, P.nbr,
                                  (const float*)P.cpl, (const float*)P.mat, nullptr, nullptr, (const float*)P.b,
                                  (float*)P.x, (float*)P.r, wsm);
  }
}

// r_c = I^T r on coarse element C by one warp (the sums of restrict_coarse,
// in the same order)
__device__ __forceinline__ void warp_restrict(int d, int s, int nb, int nc0, int nc1, int nf0, int nf1, int64_t C,
                                              const float* __restrict__ P, const float* r, float* rc, float* rs,
                                              int lane) {
  const int nch = 1 << d;
  const int I0 = (int)(C % nc0), I1 = (int)((C / nc0) % nc1), I2 = (int)(C / ((int64_t)nc0 * nc1));
  __syncwarp();
  for (int i = lane; i < nch * nb; i += 32) {
    const int ch = i / nb, k = i - ch * nb;
    const int f0 = 2 * I0 + (ch & 1), f1 = 2 * I1 + ((ch >> 1) & 1), f2 = 2 * I2 + ((ch >> 2) & 1);
    const int64_t f = (d == 2) ? f0 + (int64_t)nf0 * f1 : f0 + (int64_t)nf0 * (f1 + (int64_t)nf1 * f2);
    rs[i] = r[f * nb + k];
  }
  __syncwarp();
  for (int o = lane; o < nb; o += 32) {
    const int v = o / s, bm = o - v * s;
    float acc = 0;
    for (int ch = 0; ch < nch; ++ch) {
      const float* pc = P + ch * s * s + bm;
      const float* rr = rs + ch * nb + v * s;
      for (int a = 0; a < s; ++a) acc += pc[a * s] * rr[a];
    }
    rc[C * nb + o] = acc;
  }
  __syncwarp();
}

// x += I x_c on the children of C by one warp (the sums of prolong_coarse)
__device__ __forceinline__ void warp_prolong(int d, int s, int nb, int nf0, int nf1, int nc0, int nc1, int64_t C,
                                             const float* __restrict__ PT, const float* xc, float* x, float* xs,
                                             int lane) {
  const int nch = 1 << d;
  const int I0 = (int)(C % nc0), I1 = (int)((C / nc0) % nc1), I2 = (int)(C / ((int64_t)nc0 * nc1));
  __syncwarp();
  for (int i = lane; i < nb; i += 32) xs[i] = xc[C * nb + i];
  __syncwarp();
  for (int o = lane; o < nch * nb; o += 32) {
    const int ch = o / nb, va = o - ch * nb;
    const int v = va / s, am = va - v * s;
    const int f0 = 2 * I0 + (ch & 1), f1 = 2 * I1 + ((ch >> 1) & 1), f2 = 2 * I2 + ((ch >> 2) & 1);
    const int64_t f = (d == 2) ? f0 + (int64_t)nf0 * f1 : f0 + (int64_t)nf0 * (f1 + (int64_t)nf1 * f2);
    const float* pc = PT + ch * s * s + am;
    const float* xv = xs + v * s;
    float acc = 0;
    for (int bm = 0; bm < s; ++bm) acc += pc[bm * s] * xv[bm];
    x[f * nb + va] += acc;
  }
  __syncwarp();
}

__device__ __forceinline__ void batch_unit(const BatchProblem& B, const CyclePhase& P, int64_t v, int it, double rtol,
                                           void* wsm, int lane) {
  const Pattern& pat = B.pat;
  const int d = pat.d, s = pat.s, nb = pat.nb;
  switch (P.op) {
    case PHASE_GS:
    case PHASE_RESID:
    case PHASE_RESID64: {
      const int pos = P.pos0 + (int)v;
      switch (s) {
        case 4: batch_element<4>(pat, P.op, P, pos, wsm); break;
        case 8: batch_element<8>(pat, P.op, P, pos, wsm); break;
        case 9: batch_element<9>(pat, P.op, P, pos, wsm); break;
        case 16: batch_element<16>(pat, P.op, P, pos, wsm); break;
        case 27: batch_element<27>(pat, P.op, P, pos, wsm); break;
        default: break;
      }
      break;
    }
    case PHASE_RESTRICT:
      warp_restrict(d, s, nb, P.dims[0], P.dims[1], P.dims[2], P.dims[3], v, (const float*)P.tr, (const float*)P.in,
                    (float*)P.out, (float*)wsm, lane);
      for (int i = lane; i < nb; i += 32) ((float*)P.xz)[v * nb + i] = 0.f;
      break;
    case PHASE_PROLONG:
      warp_prolong(d, s, nb, P.dims[0], P.dims[1], P.dims[2], P.dims[3], v, (const float*)P.tr, (const float*)P.in,
                   (float*)P.out, (float*)wsm, lane);
      break;
    case PHASE_BOTTOM: {   // x = A_c^+ b, one row, FP64 accumulation (as bottom_kernel)
      const int64_t row = v;
      if (row < P.n) {
        const double* pinv = (const double*)P.tr;
        const float* bb = (const float*)P.in;
        double acc = 0.0;
        for (int64_t j = lane; j < P.n; j += 32) acc += pinv[row * P.n + j] * (double)bb[j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) ((float*)P.out)[row] = (float)acc;
      }
      break;
    }
    case PHASE_CONVERT: {   // cycle right-hand side from the outer residual, zero initial guess
      const int64_t i0 = v * kBatchChunk, i1 = min(B.n0, i0 + kBatchChunk);
      const double* r = (const double*)P.in;
      for (int64_t i = i0 + lane; i < i1; i += 32) {
        ((float*)P.out)[i] = (float)r[i];
        ((float*)P.xz)[i] = 0.f;
      }
      break;
    }
    case PHASE_AXPY: {      // x += c (the cycle's FP32 correction into the FP64 iterate)
      const int64_t i0 = v * kBatchChunk, i1 = min(B.n0, i0 + kBatchChunk);
      const float* c = (const float*)P.in;
      for (int64_t i = i0 + lane; i < i1; i += 32) ((double*)P.out)[i] += (double)c[i];
      break;
    }
    case PHASE_NORM: {      // partial sum of squares of one chunk, fixed reduction order
      const int64_t i0 = v * kBatchChunk, i1 = min(B.n0, i0 + kBatchChunk);
      const double* r = (const double*)P.in;
      double acc = 0.0;
      for (int64_t i = i0 + lane; i < i1; i += 32) acc += r[i] * r[i];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) B.part[v] = acc;
      break;
    }
    case PHASE_CHECK: {     // ||r|| / ||b|| after this iteration; stop when converged or diverged
      if (lane == 0) {
        const int64_t nch = (B.n0 + kBatchChunk - 1) / kBatchChunk;
        double sum = 0.0;
        for (int64_t c = 0; c < nch; ++c) sum += *((volatile double*)&B.part[c]);
        const double rel = sqrt(sum) / B.bnorm;
        B.hist[it + 1] = rel;
        *B.iters = it + 1;
        if (rel <= rtol) {
          *((volatile int*)B.active) = 0;
        } else if (!isfinite(rel) || rel > 1e6 * B.rel0) {
          *B.status = -5;   // STK_ERR_DIVERGED
          *((volatile int*)B.active) = 0;
        }
      }
      __syncwarp();
      break;
    }
    default: break;
  }
}

// Every outer iteration of every problem of the batch in one cooperative
// launch: x <- x + V(0, b - A x) with the V-cycle in FP32 records, the
// residual in FP64; the steps of one iteration run in order with a grid
// barrier after each; a problem whose residual reached rtol stops taking part.
__global__ void __launch_bounds__(kWideNT, 3) batch_solve_kernel(const BatchProblem* __restrict__ probs, int nprob,
                                                              const BatchStep* __restrict__ steps, int nsteps,
                                                              const BatchTask* __restrict__ tasks, int maxit,
                                                              double rtol, int slice, GridBarrierWords* gb, int* err,
                                                              long long limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_any;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  void* wsm = smem_raw + (size_t)warp * slice;
  const int64_t gw = (int64_t)blockIdx.x * wpb + warp, nw = (int64_t)gridDim.x * wpb;
  for (int it = 0; it < maxit; ++it) {
    for (int k = 0; k < nsteps; ++k) {
      const BatchStep stp = steps[k];
      int t = stp.t0;
      for (int64_t u = gw; u < stp.units; u += nw) {
        while (t + 1 < stp.t1 && tasks[t + 1].ustart <= u) ++t;
        const BatchProblem& B = probs[tasks[t].prob];
        if (*((volatile int*)B.active) == 0) continue;
        const CyclePhase P = tasks[t].ph;
        batch_unit(B, P, u - tasks[t].ustart, it, rtol, wsm, lane);
      }
      if (!grid_barrier(gb, err, limit)) return;
    }
    if (threadIdx.x == 0) {
      int any = 0;
      for (int q = 0; q < nprob; ++q) any |= *((volatile int*)probs[q].active);
      s_any = any;
    }
    __syncthreads();
    if (!s_any) return;
  }
}

}  // namespace

// Shared bytes of one warp's slice in the persistent batch.
size_t batch_smem_bytes(const Pattern& pat) {
  const WarpGeom<float> w32 = warp_geometry<float>(pat);
  const WarpGeom<double> w64 = warp_geometry<double>(pat);
  size_t slice = std::max((size_t)w32.words * sizeof(float), (size_t)w64.words * sizeof(double));
  slice = std::max(slice, (size_t)(1 << pat.d) * pat.nb * sizeof(float));
  return (slice + 15) / 16 * 16;
}

cudaError_t launch_batch_solve(const BatchProblem* probs, int nprob, const BatchStep* steps, int nsteps,
                               const BatchTask* tasks, int maxit, double rtol, int smax, size_t smem,
                               GridBarrierWords* gb, int* err, long long limit, int grid, cudaStream_t st) {
  (void)smax;
  const int slice = (int)smem;                 // per warp
  smem = (size_t)slice * (kWideNT / 32);       // per CTA
  if (smem > 226 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(batch_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0, dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_solve_kernel, kWideNT, smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidValue;
  grid = std::min(grid, per_sm * sms);
  if (grid < 1) return cudaErrorInvalidValue;
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
  return cudaLaunchKernelEx(&cfg, batch_solve_kernel, probs, nprob, steps, nsteps, tasks, maxit, rtol, slice, gb, err,
                            limit);
}

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
