// Per-element device code shared by the element kernels (kernels.cu) and the
// persistent coarse-cycle kernel (persist.cu): the storage precisions of the
// element records, the one-CTA-per-element colour step / residual, and the
// transfers of one coarse element.  Both translation units run these bodies,
// so a step gives the same bits in either.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "stk_internal.h"

namespace stk {

template <typename TS> struct StorageTraits;
template <> struct StorageTraits<double> {
  using Acc = double;
  static constexpr int V = 2;
  __device__ static inline void load(const double* p, double* w) {
    double2 v = __ldcs(reinterpret_cast<const double2*>(p));
    w[0] = v.x;
    w[1] = v.y;
  }
  __device__ static inline void load_keep(const double* p, double* w) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    w[0] = v.x;
    w[1] = v.y;
  }
  __device__ static inline void load_shared(const double* p, double* w) {
    double2 v = *reinterpret_cast<const double2*>(p);
    w[0] = v.x;
    w[1] = v.y;
  }
};
template <> struct StorageTraits<float> {
  using Acc = float;
  static constexpr int V = 4;
  __device__ static inline void load(const float* p, float* w) {
    float4 v = __ldcs(reinterpret_cast<const float4*>(p));
    w[0] = v.x;
    w[1] = v.y;
    w[2] = v.z;
    w[3] = v.w;
  }
  __device__ static inline void load_keep(const float* p, float* w) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    w[0] = v.x;
    w[1] = v.y;
    w[2] = v.z;
    w[3] = v.w;
  }
  __device__ static inline void load_shared(const float* p, float* w) {
    float4 v = *reinterpret_cast<const float4*>(p);
    w[0] = v.x;
    w[1] = v.y;
    w[2] = v.z;
    w[3] = v.w;
  }
};
template <> struct StorageTraits<__nv_bfloat16> {
  using Acc = float;
  static constexpr int V = 8;
  __device__ static inline void load(const __nv_bfloat16* p, float* w) {
    uint4 v = __ldcs(reinterpret_cast<const uint4*>(p));
    uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      w[2 * i] = __uint_as_float(u[i] << 16);
      w[2 * i + 1] = __uint_as_float(u[i] & 0xffff0000u);
    }
  }
  __device__ static inline void load_keep(const __nv_bfloat16* p, float* w) {
    uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      w[2 * i] = __uint_as_float(u[i] << 16);
      w[2 * i + 1] = __uint_as_float(u[i] & 0xffff0000u);
    }
  }
  __device__ static inline void load_shared(const __nv_bfloat16* p, float* w) {
    uint4 v = *reinterpret_cast<const uint4*>(p);
    uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      w[2 * i] = __uint_as_float(u[i] << 16);
      w[2 * i + 1] = __uint_as_float(u[i] & 0xffff0000u);
    }
  }
};

// FP16 records carry a power-of-two scale per coupling sub-block and per row
// of the dense blocks (applied in the row sums, see element_warp_kernel).
template <> struct StorageTraits<__half> {
  using Acc = float;
  static constexpr int V = 8;
  __device__ static inline void cvt(uint4 v, float* w) {
    const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      w[2 * i] = __half2float(__ushort_as_half((unsigned short)(u[i] & 0xffffu)));
      w[2 * i + 1] = __half2float(__ushort_as_half((unsigned short)(u[i] >> 16)));
    }
  }
  __device__ static inline void load(const __half* p, float* w) { cvt(__ldcs(reinterpret_cast<const uint4*>(p)), w); }
  __device__ static inline void load_keep(const __half* p, float* w) {
    cvt(__ldg(reinterpret_cast<const uint4*>(p)), w);
  }
  __device__ static inline void load_shared(const __half* p, float* w) {
    cvt(*reinterpret_cast<const uint4*>(p), w);
  }
};

template <typename TS>
constexpr bool kScaledStorage = std::is_same<TS, __half>::value;

__host__ __device__ inline int task_scale_stride(const Pattern& pat) { return (pat.T + 3) / 4 * 4; }

// ---- one CTA per element (latency variant for launches of few elements) ------
constexpr int kWideNT = 256;

struct WideGeom {
  int CGc, KC;   // coupling column groups and columns per group
  int NCG, CW;   // dense column groups and columns per group
  int XS;        // gathered slot stride
  size_t words;  // accumulator words of shared memory (after the index block)
  // the element's records staged in shared memory by cp.async (when they fit):
  // byte offset of the staging area, its size, and 1 when staging is used
  size_t rec_off, rec_bytes;
  int prefetch;
};

constexpr size_t kWideStageBudget = 96 * 1024;   // shared bytes per CTA above which records are not staged

// Shared bytes one CTA of the one-CTA-per-element body needs.
__host__ __device__ inline size_t wide_smem_bytes(const WideGeom& g) {
  return g.prefetch ? g.rec_off + g.rec_bytes : g.rec_off;
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned int d = (unsigned int)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Programmatic dependent launch: a kernel lets the next launch on its stream
// start (griddepcontrol.launch_dependents; a no-op when that launch does not
// ask for it), and a kernel launched with programmatic serialisation waits
// for the previous one to complete, its writes visible, before it touches
// what that kernel may write (griddepcontrol.wait; a no-op otherwise).
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename TS>
__host__ __device__ inline WideGeom wide_geometry(const Pattern& pat) {
  constexpr int V = StorageTraits<TS>::V;
  WideGeom g;
  const int nvr = pat.TRP / V;
  g.CGc = nvr > 0 ? kWideNT / nvr : 1;
  if (g.CGc < 1) g.CGc = 1;
  if (g.CGc > pat.s) g.CGc = pat.s;
  g.KC = (pat.s + g.CGc - 1) / g.CGc;
  const int NRV = pat.NBP / V;
  g.NCG = kWideNT / NRV;
  if (g.NCG < 1) g.NCG = 1;
  if (g.NCG > pat.nb) g.NCG = pat.nb;
  g.CW = (pat.nb + g.NCG - 1) / g.NCG;
  g.XS = pat.s + 1;
  g.words = (size_t)pat.NG * g.XS + (size_t)g.CGc * pat.TRP + 2 * (size_t)pat.NBP + (size_t)g.NCG * pat.NBP;
  if (kScaledStorage<TS>) g.words += task_scale_stride(pat);
  using TA = typename StorageTraits<TS>::Acc;
  g.rec_off = (kMaxOffsets * sizeof(int) + g.words * sizeof(TA) + 15) / 16 * 16;
  g.rec_bytes = ((size_t)pat.s * pat.TRP + (size_t)pat.nb * pat.NBP) * sizeof(TS);
  g.prefetch = g.rec_off + g.rec_bytes <= kWideStageBudget ? 1 : 0;
  return g;
}

// Start copying element pos's coupling record and dense block (A_ii^{-1} or
// A_ii) into the CTA's staging area; they do not depend on x, so the copy
// overlaps the neighbour gather (and, in the persistent cycle, the grid
// barrier before the phase).  Records are 16-byte aligned: TRP and NBP are
// multiples of 8 entries.
template <typename TS>
__device__ __forceinline__ void wide_stage(const Pattern& pat, const WideGeom& wg, int pos, const TS* cpl,
                                           const TS* mat, unsigned char* smem_raw) {
  unsigned char* dst = smem_raw + wg.rec_off;
  const size_t cb = (size_t)pat.s * pat.TRP * sizeof(TS), mb = (size_t)pat.nb * pat.NBP * sizeof(TS);
  const unsigned char* c0 = reinterpret_cast<const unsigned char*>(cpl + (size_t)pos * pat.s * pat.TRP);
  const unsigned char* m0 = reinterpret_cast<const unsigned char*>(mat + (size_t)pos * pat.nb * pat.NBP);
  for (size_t i = (size_t)threadIdx.x * 16; i < cb; i += (size_t)blockDim.x * 16) cp_async16(dst + i, c0 + i);
  for (size_t i = (size_t)threadIdx.x * 16; i < mb; i += (size_t)blockDim.x * 16) cp_async16(dst + cb + i, m0 + i);
  cp_async_commit();
}

// One element (position pos) of a colour step (MODE_GS) or residual
// (MODE_RESID) by one CTA of kWideNT threads: every (task-row vector, column
// group) and (row vector, column group) pair of the element in flight at once,
// records read with L2-keeping loads.  smem_raw: the CTA's dynamic shared
// memory (kMaxOffsets ints, then wg.words accumulators).  Starts and ends with
// all threads of the CTA in step.  b, x and rout carry no __restrict__: in the
// persistent cycle earlier phases of the same launch write them, so their
// loads must not take the read-only (non-coherent) path.
template <typename TS, typename TX, int S, bool ST>
__device__ __forceinline__ void wide_element_impl(const Pattern& pat, const WideGeom& wg, int mode, int pos,
                                                  const int* __restrict__ perm, const int* __restrict__ nbr,
                                                  const TS* __restrict__ cpl, const TS* __restrict__ mat,
                                                  const float* __restrict__ tsc, const float* __restrict__ rsc,
                                                  const TX* b, TX* x, TX* rout, unsigned char* smem_raw,
                                                  bool staged) {
  using Tr = StorageTraits<TS>;
  using TA = typename Tr::Acc;
  constexpr int V = Tr::V;
  const int nb = pat.nb, NBP = pat.NBP, TRP = pat.TRP, TR = pat.TR;
  const int NRV = NBP / V, nvr = TRP / V;
  const int TP = task_scale_stride(pat);

  int* nbs = reinterpret_cast<int*>(smem_raw);   // kMaxOffsets neighbour indices
  TA* Xs = reinterpret_cast<TA*>(smem_raw + kMaxOffsets * sizeof(int));
  TA* part = Xs + pat.NG * wg.XS;
  TA* g = part + wg.CGc * TRP;
  TA* xi = g + NBP;
  TA* part2 = xi + NBP;
  TA* tss = part2 + wg.NCG * NBP;   // task scales (FP16 records only)

  const int tid = threadIdx.x;
  if (ST && !staged) wide_stage<TS>(pat, wg, pos, cpl, mat, smem_raw);
  const int e = perm[pos];
  for (int i = tid; i < pat.NO; i += kWideNT) nbs[i] = nbr[(size_t)pos * pat.NO + i];
  for (int i = tid; i < nb; i += kWideNT) {
    g[i] = (TA)b[(size_t)e * nb + i];
    if (mode == MODE_RESID) xi[i] = (TA)x[(size_t)e * nb + i];
  }
  if constexpr (kScaledStorage<TS>)
    for (int i = tid; i < pat.T; i += kWideNT) tss[i] = tsc[(size_t)pos * TP + i];
  __syncthreads();
  for (int i = tid; i < pat.NG * S; i += kWideNT) {
    const int gi = i / S, ci = i - gi * S;
    const int j = nbs[pat.g_o[gi]];
    Xs[gi * wg.XS + ci] = (j >= 0) ? (TA)x[(size_t)j * nb + pat.g_cv[gi] * S + ci] : (TA)0;
  }
  __syncthreads();
  if (ST) {
    cp_async_wait_all();
    __syncthreads();
  }
  const TS* rec = ST ? reinterpret_cast<const TS*>(smem_raw + wg.rec_off) : cpl + (size_t)pos * S * TRP;
  for (int u = tid; u < nvr * wg.CGc; u += kWideNT) {
    const int tv = u % nvr, cg = u / nvr;
    const int c0 = cg * wg.KC, c1 = min(S, c0 + wg.KC);
    const int tr0 = tv * V;
    const TA* xp[V];
    TA acc[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const int tr = tr0 + j;
      xp[j] = (tr < TR) ? Xs + pat.task_g[tr / S] * wg.XS : Xs;
      acc[j] = 0;
    }
#pragma unroll 8
    for (int ci = c0; ci < c1; ++ci) {
      TA w[V];
      if (ST)
        Tr::load_shared(rec + (size_t)ci * TRP + tr0, w);
      else
        Tr::load_keep(rec + (size_t)ci * TRP + tr0, w);
#pragma unroll
      for (int j = 0; j < V; ++j) acc[j] = fma(w[j], xp[j][ci], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < V; ++j) part[cg * TRP + tr0 + j] = acc[j];
  }
  __syncthreads();
  for (int r = tid; r < nb; r += kWideNT) {
    const int rv = r / S, rr = r - rv * S;
    TA sum = 0;
    for (int t = pat.rv_t0[rv]; t < pat.rv_t1[rv]; ++t) {
      TA st = 0;
      for (int cg = 0; cg < wg.CGc; ++cg) st += part[cg * TRP + t * S + rr];
      if constexpr (kScaledStorage<TS>) st *= tss[t];
      sum += st;
    }
    g[r] = g[r] - sum;
  }
  __syncthreads();
  const TS* mrec = ST ? rec + (size_t)S * TRP : mat + (size_t)pos * nb * NBP;
  const TA* vin = (mode == MODE_GS) ? g : xi;
  for (int u = tid; u < NRV * wg.NCG; u += kWideNT) {
    const int rvv = u % NRV, cg = u / NRV;
    const int c0 = cg * wg.CW, c1 = min(nb, c0 + wg.CW);
    TA acc[V];
#pragma unroll
    for (int j = 0; j < V; ++j) acc[j] = 0;
#pragma unroll 4
    for (int ci = c0; ci < c1; ++ci) {
      TA w[V];
      if (ST)
        Tr::load_shared(mrec + (size_t)ci * NBP + rvv * V, w);
      else
        Tr::load_keep(mrec + (size_t)ci * NBP + rvv * V, w);
      const TA v = vin[ci];
#pragma unroll
      for (int j = 0; j < V; ++j) acc[j] = fma(w[j], v, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < V; ++j) part2[cg * NBP + rvv * V + j] = acc[j];
  }
  __syncthreads();
  for (int r = tid; r < nb; r += kWideNT) {
    TA sum = 0;
    for (int cg = 0; cg < wg.NCG; ++cg) sum += part2[cg * NBP + r];
    if constexpr (kScaledStorage<TS>) sum *= rsc[(size_t)pos * NBP + r];
    if (mode == MODE_GS)
      x[(size_t)e * nb + r] = (TX)sum;
    else
      rout[(size_t)e * nb + r] = (TX)(g[r] - sum);
  }
  __syncthreads();
}

// The element body with or without staging its records (wg.prefetch; same
// arithmetic, same bits).  staged: the caller already issued wide_stage for
// this pos (the persistent cycle does so before its grid barrier).
template <typename TS, typename TX, int S>
__device__ __forceinline__ void wide_element(const Pattern& pat, const WideGeom& wg, int mode, int pos,
                                             const int* __restrict__ perm, const int* __restrict__ nbr,
                                             const TS* __restrict__ cpl, const TS* __restrict__ mat,
                                             const float* __restrict__ tsc, const float* __restrict__ rsc,
                                             const TX* b, TX* x, TX* rout, unsigned char* smem_raw,
                                             bool staged = false) {
  if (wg.prefetch)
    wide_element_impl<TS, TX, S, true>(pat, wg, mode, pos, perm, nbr, cpl, mat, tsc, rsc, b, x, rout, smem_raw,
                                       staged);
  else
    wide_element_impl<TS, TX, S, false>(pat, wg, mode, pos, perm, nbr, cpl, mat, tsc, rsc, b, x, rout, smem_raw,
                                        false);
}

// ---- one warp per element (the bandwidth kernel of large launches) ------------
constexpr int kWarps = 8;   // warps per CTA of element_warp_kernel

template <typename TS>
struct WarpGeom {
  int NCG, CW, XS, words;  // column groups, columns per group, X slot stride, TA words per warp
};

template <typename TS>
__host__ __device__ inline WarpGeom<TS> warp_geometry(const Pattern& pat) {
  constexpr int V = StorageTraits<TS>::V;
  WarpGeom<TS> g;
  const int NRV = pat.NBP / V;
  g.NCG = (32 / NRV) > 0 ? (32 / NRV) : 1;
  g.CW = (pat.nb + g.NCG - 1) / g.NCG;
  g.XS = pat.s + 1;
  int w = pat.NG * g.XS + pat.TRP + 2 * pat.NBP + g.NCG * pat.NBP;
  if (kScaledStorage<TS>) w += task_scale_stride(pat);
  g.words = (w + 3) / 4 * 4;
  return g;
}

// One element (position pos) of a colour step (MODE_GS) or residual
// (MODE_RESID) by one warp: the gathered neighbour values and partial sums in
// the warp's own shared-memory slice (wg.words accumulators), each lane
// streaming V consecutive task-rows column by column with 16-byte evict-first
// loads, then the dense block in column groups; only __syncwarp.  b, x and
// rout carry no __restrict__ (the persistent batch writes them in earlier
// steps of the same launch).
template <typename TS, typename TX, int S>
__device__ __forceinline__ void warp_element(const Pattern& pat, const WarpGeom<TS>& wg, int mode, int pos,
                                             const int* __restrict__ perm, const int* __restrict__ nbr,
                                             const TS* __restrict__ cpl, const TS* __restrict__ mat,
                                             const float* __restrict__ tsc, const float* __restrict__ rsc,
                                             const TX* b, TX* x, TX* rout, void* warp_smem) {
  using Tr = StorageTraits<TS>;
  using TA = typename Tr::Acc;
  constexpr int V = Tr::V;
  const int nb = pat.nb, NBP = pat.NBP, TRP = pat.TRP, TR = pat.TR;
  const int NRV = NBP / V;
  const int TP = task_scale_stride(pat);
  const int lane = threadIdx.x & 31;
  TA* base = reinterpret_cast<TA*>(warp_smem);
  TA* Xs = base;
  TA* part = Xs + pat.NG * wg.XS;
  TA* g = part + TRP;
  TA* xi = g + NBP;
  TA* part2 = xi + NBP;
  TA* tss = part2 + wg.NCG * NBP;   // task scales (FP16 records only)

  const int e = perm[pos];
  const int* nbe = nbr + (size_t)pos * pat.NO;
  for (int i = lane; i < pat.NG * S; i += 32) {
    const int gi = i / S, ci = i - gi * S;
    const int j = nbe[pat.g_o[gi]];
    Xs[gi * wg.XS + ci] = (j >= 0) ? (TA)x[(size_t)j * nb + pat.g_cv[gi] * S + ci] : (TA)0;
  }
  for (int i = lane; i < nb; i += 32) {
    g[i] = (TA)b[(size_t)e * nb + i];
    if (mode == MODE_RESID) xi[i] = (TA)x[(size_t)e * nb + i];
  }
  if constexpr (kScaledStorage<TS>)
    for (int i = lane; i < pat.T; i += 32) tss[i] = tsc[(size_t)pos * TP + i];
  __syncwarp();
  const TS* rec = cpl + (size_t)pos * S * TRP;
  for (int tv = lane; tv < TRP / V; tv += 32) {
    const int tr0 = tv * V;
    const TA* xp[V];
    TA acc[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const int tr = tr0 + j;
      xp[j] = (tr < TR) ? Xs + pat.task_g[tr / S] * wg.XS : Xs;
      acc[j] = 0;
    }
#pragma unroll
    for (int ci = 0; ci < S; ++ci) {
      TA w[V];
      Tr::load(rec + (size_t)ci * TRP + tr0, w);
#pragma unroll
      for (int j = 0; j < V; ++j) acc[j] = fma(w[j], xp[j][ci], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < V; ++j) part[tr0 + j] = acc[j];
  }
  __syncwarp();
  for (int r = lane; r < nb; r += 32) {
    const int rv = r / S, rr = r - rv * S;
    TA sum = 0;
    if constexpr (kScaledStorage<TS>) {
      for (int t = pat.rv_t0[rv]; t < pat.rv_t1[rv]; ++t) sum += part[t * S + rr] * tss[t];
    } else {
      for (int t = pat.rv_t0[rv]; t < pat.rv_t1[rv]; ++t) sum += part[t * S + rr];
    }
    g[r] = g[r] - sum;
  }
  __syncwarp();
  const TS* mrec = mat + (size_t)pos * nb * NBP;
  const TA* vin = (mode == MODE_GS) ? g : xi;
  // row scales of the FP16 dense block, fetched before its loads (nb <= 128)
  float rs[4] = {1.f, 1.f, 1.f, 1.f};
  if constexpr (kScaledStorage<TS>) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (lane + 32 * q < nb) rs[q] = rsc[(size_t)pos * NBP + lane + 32 * q];
  }
  for (int u = lane; u < NRV * wg.NCG; u += 32) {
    const int rvv = u % NRV, cg = u / NRV;
    const int c0 = cg * wg.CW, c1 = min(nb, c0 + wg.CW);
    TA acc[V];
#pragma unroll
    for (int j = 0; j < V; ++j) acc[j] = 0;
#pragma unroll 4
    for (int ci = c0; ci < c1; ++ci) {
      TA w[V];
      Tr::load(mrec + (size_t)ci * NBP + rvv * V, w);
      const TA v = vin[ci];
#pragma unroll
      for (int j = 0; j < V; ++j) acc[j] = fma(w[j], v, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < V; ++j) part2[cg * NBP + rvv * V + j] = acc[j];
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = lane + 32 * q;
    if (r >= nb) break;
    TA sum = 0;
    for (int cg = 0; cg < wg.NCG; ++cg) sum += part2[cg * NBP + r];
    if constexpr (kScaledStorage<TS>) sum *= rs[q];
    if (mode == MODE_GS)
      x[(size_t)e * nb + r] = (TX)sum;
    else
      rout[(size_t)e * nb + r] = (TX)(g[r] - sum);
  }
  __syncwarp();
}

// ---- restriction / prolongation of one coarse element -------------------------
// P[ch][a][b]: fine coefficient a of coarse mode b for child ch (P_f of the
// scalar injection; the (d+1) variables share it).  One CTA per coarse
// element: the children's residual blocks (restriction) or the coarse block
// (prolongation) are staged in shared memory (rs / xs: 2^d nb entries) with
// coalesced loads; arithmetic is in the vector precision TX.  The vectors carry
// no __restrict__ (the persistent cycle writes them in earlier phases).
template <typename TX>
__device__ __forceinline__ void restrict_coarse(int d, int s, int nb, int nc0, int nc1, int nf0, int nf1, int64_t C,
                                                const TX* __restrict__ P, const TX* r, TX* rc, TX* rs) {
  const int nch = 1 << d;
  const TX* Ps = P;   // small, read through the read-only cache
  const int I0 = (int)(C % nc0), I1 = (int)((C / nc0) % nc1), I2 = (int)(C / ((int64_t)nc0 * nc1));
  __syncthreads();
  for (int i = threadIdx.x; i < nch * nb; i += blockDim.x) {
    const int ch = i / nb, k = i - ch * nb;
    const int f0 = 2 * I0 + (ch & 1), f1 = 2 * I1 + ((ch >> 1) & 1), f2 = 2 * I2 + ((ch >> 2) & 1);
    const int64_t f = (d == 2) ? f0 + (int64_t)nf0 * f1 : f0 + (int64_t)nf0 * (f1 + (int64_t)nf1 * f2);
    rs[i] = r[f * nb + k];
  }
  __syncthreads();
  for (int o = threadIdx.x; o < nb; o += blockDim.x) {
    const int v = o / s, bm = o - v * s;
    TX acc = 0;
    for (int ch = 0; ch < nch; ++ch) {
      const TX* pc = Ps + ch * s * s + bm;
      const TX* rr = rs + ch * nb + v * s;
      for (int a = 0; a < s; ++a) acc += pc[a * s] * rr[a];
    }
    rc[C * nb + o] = acc;
  }
}

// PT[ch][b][a] = P[ch][a][b]; x (fine) += I x_c on the children of C.
template <typename TX>
__device__ __forceinline__ void prolong_coarse(int d, int s, int nb, int nf0, int nf1, int nc0, int nc1, int64_t C,
                                               const TX* __restrict__ PT, const TX* xc, TX* x, TX* xs) {
  const int nch = 1 << d;
  const TX* Ps = PT;  // small, read through the read-only cache
  const int I0 = (int)(C % nc0), I1 = (int)((C / nc0) % nc1), I2 = (int)(C / ((int64_t)nc0 * nc1));
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x) xs[i] = xc[C * nb + i];
  __syncthreads();
  for (int o = threadIdx.x; o < nch * nb; o += blockDim.x) {
    const int ch = o / nb, va = o - ch * nb;
    const int v = va / s, am = va - v * s;
    const int f0 = 2 * I0 + (ch & 1), f1 = 2 * I1 + ((ch >> 1) & 1), f2 = 2 * I2 + ((ch >> 2) & 1);
    const int64_t f = (d == 2) ? f0 + (int64_t)nf0 * f1 : f0 + (int64_t)nf0 * (f1 + (int64_t)nf1 * f2);
    const TX* pc = Ps + ch * s * s + am;
    const TX* xv = xs + v * s;
    TX acc = 0;
    for (int bm = 0; bm < s; ++bm) acc += pc[bm * s] * xv[bm];
    x[f * nb + va] += acc;
  }
}

}  // namespace stk
