// Kernels of general block-sparse levels (the cut-cell hierarchy): the
// coloured block Gauss-Seidel step and the residual of Section 3 with
// per-element coupling lists of any length, and the transfers of Algorithm 1
// through per-element injection blocks.
//
// Element kernel: W warps per element position of the launch (W by launch
// size).  Task t of the element is one s x s sub-block C_t (row variable rv,
// column variable cv, neighbour j), stored row-major, 16 x 16 for p = 3.  Lane pair
// (2r, 2r+1) owns row r: each lane multiplies half the row with the matching
// half of x_j (16-byte loads of records and vector), the pair sums with one
// shuffle and adds the result into the running sum of row r of variable rv.
// A task's record is one contiguous 1 KB (FP32) read by the whole warp.  The
// dense A_ii^{-1} (colour step) or A_ii (residual) is stored column-major,
// nb columns of nbp rows (nbp: nb rounded up to 16 bytes of entries), and
// staged in shared memory.
#include <cuda_runtime.h>

#include "element_core.cuh"
#include "stk_internal.h"
#include "../../include/stokes_mg.h"

namespace stk {

namespace {

constexpr int kGenWarps = 4;    // warps (elements) per CTA
constexpr int kGenMaxNb = 64;   // largest block (2D, p = 3: 3 x 16)

template <typename T, typename V, int N>
__device__ __forceinline__ V dot_n(const T* __restrict__ a, const V* b) {
  V acc = V(0);
#pragma unroll
  for (int k = 0; k < N; ++k) acc += (V)a[k] * b[k];
  return acc;
}

__device__ __forceinline__ void gen_cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned int d = (unsigned int)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void gen_cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void gen_cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Half a row of a 16-column block: 8 entries from 16-byte aligned addresses.
__device__ __forceinline__ void load8(const float* p, float* v) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p)), b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void load8(const double* p, double* v) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p) + k);
    v[2 * k] = a.x;
    v[2 * k + 1] = a.y;
  }
}
// The iterate is written by other launches (and, for the element's own block,
// by this one), so it is read through plain loads.
__device__ __forceinline__ void load8v(const float* p, float* v) {
  const float4 a = *reinterpret_cast<const float4*>(p), b = *(reinterpret_cast<const float4*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void load8v(const double* p, double* v) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 a = *(reinterpret_cast<const double2*>(p) + k);
    v[2 * k] = a.x;
    v[2 * k + 1] = a.y;
  }
}

// W warps per element (W = 1, 2, 4; 4 / W elements per CTA of 4 warps): warp
// wi of an element takes the wi-th contiguous chunk of its tasks, the row sums
// of the W warps meet in shared memory, and the element's W x 32 threads share
// the dense product by rows.  The element's dense block (A_ii^{-1} or A_ii) is
// copied into shared memory by cp.async when the kernel starts, so that its
// load overlaps the coupling tasks and the dense product reads shared memory.
// Small launches (the coarse levels) take W = 4, so that each element's chain
// of dependent record rounds is a quarter as long; larger ones W = 2.
template <typename T, typename V, int S, int MODE, int W>
__global__ void __launch_bounds__(kGenWarps * 32, 6)
    gen_element_kernel(int pos0, int npos, int nb, int nbp, const int* __restrict__ perm,
                       const int* __restrict__ tptr, const int* __restrict__ tinfo, const T* __restrict__ cpl,
                       const T* __restrict__ mat, const V* b, V* x, V* r) {
  constexpr int H = (S + 1) / 2;   // columns of the first half-row
  constexpr int G = 32 * W;        // threads per element
  constexpr int E = kGenWarps / W; // elements per CTA
  __shared__ V part[kGenWarps][3][16];
  __shared__ V sg[E][kGenMaxNb];
  __shared__ V sx[E][kGenMaxNb];
  extern __shared__ __align__(16) unsigned char gen_dyn[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = threadIdx.x / G, gt = threadIdx.x % G, wi = gt >> 5;
  const int pos = pos0 + blockIdx.x * E + grp;
  const bool valid = pos < pos0 + npos;   // uniform over the element's warps
  pdl_trigger();   // the next launch may start
  const int e = valid ? perm[pos] : 0;
  // the dense block, nb x nbp entries (nbp a multiple of 16 bytes), staged
  T* smat = reinterpret_cast<T*>(gen_dyn) + (size_t)grp * nb * nbp;
  if (valid) {
    const int chunks = nb * nbp * (int)sizeof(T) / 16;
    const unsigned char* src = reinterpret_cast<const unsigned char*>(mat + (size_t)pos * nb * nbp);
    for (int q = gt; q < chunks; q += G)
      gen_cp_async16(reinterpret_cast<unsigned char*>(smat) + (size_t)q * 16, src + (size_t)q * 16);
  }
  gen_cp_async_commit();
  const int row = lane >> 1, half = lane & 1;
  const bool active = row < S;
  const int c0 = half ? H : 0;
  V acc0 = V(0), acc1 = V(0), acc2 = V(0);
  int t = 0, t1 = 0;
  if (valid) {
    const int a0 = tptr[pos], a1 = tptr[pos + 1];
    const int chunk = (a1 - a0 + W - 1) / W;
    t = min(a1, a0 + wi * chunk);
    t1 = min(a1, t + chunk);
  }
  // Everything above reads what no launch writes (indices, the dense block);
  // the iterate and right-hand side wait for the previous launch.
  pdl_wait();
  auto add = [&](int rv, V pv) {
    pv += __shfl_xor_sync(0xffffffffu, pv, 1);
    if (rv == 0) acc0 += pv;
    else if (rv == 1) acc1 += pv;
    else acc2 += pv;
  };
  if (S == 16) {
    // U tasks per round (4 with FP32 records, 2 with FP64 ones, the most the
    // 80 registers hold without spilling): their words, records and x
    // segments are all requested before the first product
    constexpr int U = sizeof(T) == 4 ? 4 : 2;
    for (; t + U <= t1; t += U) {
      int info[U];
#pragma unroll
      for (int u = 0; u < U; ++u) info[u] = __ldg(tinfo + t + u);
      T a[U][8];
      V v[U][8];
      if (active) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          load8(cpl + (size_t)(t + u) * S * S + row * S + c0, a[u]);
          load8v(x + (size_t)(info[u] >> 4) * nb + (info[u] & 3) * S + c0, v[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        V pv = V(0);
        if (active)
#pragma unroll
          for (int k = 0; k < 8; ++k) pv += (V)a[u][k] * v[u][k];
        add((info[u] >> 2) & 3, pv);
      }
    }
  }
  for (; t < t1; ++t) {
    const int info = __ldg(tinfo + t);
    const int j = info >> 4, rv = (info >> 2) & 3, cv = info & 3;
    V pv = V(0);
    if (active) {
      const T* rec = cpl + (size_t)t * S * S + row * S + c0;
      const V* xj = x + (size_t)j * nb + cv * S + c0;
      if (S == 16) {
        T a[8];
        V v[8];
        load8(rec, a);
        load8v(xj, v);
#pragma unroll
        for (int k = 0; k < 8; ++k) pv += (V)a[k] * v[k];
      } else if (half) {
        pv = dot_n<T, V, S - H>(rec, xj);
      } else {
        pv = dot_n<T, V, H>(rec, xj);
      }
    }
    add(rv, pv);
  }
  if (active && !half) {
    part[w][0][row] = acc0;
    part[w][1][row] = acc1;
    part[w][2][row] = acc2;
  }
  gen_cp_async_wait_all();
  __syncthreads();
  if (valid) {
    for (int o = gt; o < nb; o += G) {
      const int v = o / S, rr = o % S;
      V sum = V(0);
#pragma unroll
      for (int q = 0; q < W; ++q) sum += part[grp * W + q][v][rr];
      sg[grp][o] = b[(size_t)e * nb + o] - sum;
      if (MODE == MODE_RESID) sx[grp][o] = x[(size_t)e * nb + o];
    }
  }
  __syncthreads();
  if (!valid) return;
  for (int o = gt; o < nb; o += G) {
    V y = V(0);
    if (MODE == MODE_GS) {
      for (int k = 0; k < nb; ++k) y += (V)smat[k * nbp + o] * sg[grp][k];
      x[(size_t)e * nb + o] = y;
    } else {
      for (int k = 0; k < nb; ++k) y += (V)smat[k * nbp + o] * sx[grp][k];
      r[(size_t)e * nb + o] = sg[grp][o] - y;
    }
  }
}

// r_c(c) = sum over children f of I_f^T r(f), per variable; one thread per
// coarse unknown.
template <typename V, typename T>
__global__ void gen_restrict_kernel(int nc, int s, int nb, const int* __restrict__ cptr,
                                    const int* __restrict__ clist, const T* __restrict__ I, const V* __restrict__ r,
                                    V* __restrict__ rc) {
  pdl_trigger();   // the next launch may start
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nc * nb) return;
  const int c = (int)(idx / nb), row = (int)(idx % nb), v = row / s, a = row % s;
  V sum = V(0);
  for (int k = cptr[c]; k < cptr[c + 1]; ++k) {
    const int f = clist[k];
    const T* If = I + (size_t)f * s * s;
    const V* rf = r + (size_t)f * nb + v * s;
    for (int bb = 0; bb < s; ++bb) sum += (V)If[bb * s + a] * rf[bb];
  }
  rc[idx] = sum;
}

// x(f) += I_f x_c(parent(f)), per variable; one thread per fine unknown.
template <typename V, typename T>
__global__ void gen_prolong_kernel(int nf, int s, int nb, const int* __restrict__ parent, const T* __restrict__ I,
                                   const V* __restrict__ xc, V* __restrict__ x) {
  pdl_trigger();   // the next launch may start
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nf * nb) return;
  const int f = (int)(idx / nb), row = (int)(idx % nb), v = row / s, a = row % s;
  const T* If = I + (size_t)f * s * s + (size_t)a * s;
  const V* xp = xc + (size_t)parent[f] * nb + v * s;
  V sum = V(0);
  for (int bb = 0; bb < s; ++bb) sum += (V)If[bb] * xp[bb];
  x[idx] += sum;
}

template <typename T, typename V, int S, int W>
cudaError_t gen_launch_w(int mode, int nb, int nbp, int pos0, int npos, const int* perm, const int* tptr,
                         const int* tinfo, const void* cpl, const void* mat, const void* b, void* x, void* r,
                         int ov, cudaStream_t st) {
  constexpr int E = kGenWarps / W;
  const int blocks = (npos + E - 1) / E;
  const size_t smem = (size_t)E * nb * nbp * sizeof(T);
  if (((size_t)nb * nbp * sizeof(T)) % 16 != 0 || smem > 200 * 1024) return cudaErrorInvalidValue;
  static bool opted[2] = {false, false};
  if (!opted[mode == MODE_GS ? 0 : 1]) {
    // the staged dense blocks of 4 / W elements (FP64 p = 3, W = 1: 72 KB)
    cudaError_t e = mode == MODE_GS
                        ? cudaFuncSetAttribute(gen_element_kernel<T, V, S, MODE_GS, W>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)
                        : cudaFuncSetAttribute(gen_element_kernel<T, V, S, MODE_RESID, W>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    opted[mode == MODE_GS ? 0 : 1] = true;
  }
  // ov: programmatic serialisation (the kernel starts during the previous
  // launch, stages its dense blocks, then waits for it before any vector)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(kGenWarps * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = ov ? 1 : 0;
  if (mode == MODE_GS)
    return cudaLaunchKernelEx(&cfg, gen_element_kernel<T, V, S, MODE_GS, W>, pos0, npos, nb, nbp, perm, tptr, tinfo,
                              (const T*)cpl, (const T*)mat, (const V*)b, (V*)x, (V*)r);
  return cudaLaunchKernelEx(&cfg, gen_element_kernel<T, V, S, MODE_RESID, W>, pos0, npos, nb, nbp, perm, tptr, tinfo,
                            (const T*)cpl, (const T*)mat, (const V*)b, (V*)x, (V*)r);
}

// Warps per element by launch size and record width (measured on the 128^2
// p = 3 cut mesh): launches of fewer than 8 (FP32) or 32 (FP64) elements per
// SM take four warps per element, larger ones two; one warp per element was
// never faster (FP64 residual of 16,468 elements: 0.406 ms with one warp,
// 0.336 with two; FP32 colour sweep 0.182 / 0.167 ms).
template <typename T, typename V, int S>
cudaError_t gen_launch(int mode, int warps, int nb, int nbp, int pos0, int npos, const int* perm, const int* tptr,
                       const int* tinfo, const void* cpl, const void* mat, const void* b, void* x, void* r, int ov,
                       cudaStream_t st) {
  if (warps == 1)
    return gen_launch_w<T, V, S, 1>(mode, nb, nbp, pos0, npos, perm, tptr, tinfo, cpl, mat, b, x, r, ov, st);
  if (warps == 2)
    return gen_launch_w<T, V, S, 2>(mode, nb, nbp, pos0, npos, perm, tptr, tinfo, cpl, mat, b, x, r, ov, st);
  if (warps == 4)
    return gen_launch_w<T, V, S, 4>(mode, nb, nbp, pos0, npos, perm, tptr, tinfo, cpl, mat, b, x, r, ov, st);
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  const int64_t four_below = (int64_t)sms * (sizeof(T) == 4 ? 8 : 32);
  if ((int64_t)npos >= four_below)
    return gen_launch_w<T, V, S, 2>(mode, nb, nbp, pos0, npos, perm, tptr, tinfo, cpl, mat, b, x, r, ov, st);
  return gen_launch_w<T, V, S, 4>(mode, nb, nbp, pos0, npos, perm, tptr, tinfo, cpl, mat, b, x, r, ov, st);
}

template <typename T, typename V>
cudaError_t gen_dispatch(int mode, int warps, int s, int nb, int nbp, int pos0, int npos, const int* perm,
                         const int* tptr, const int* tinfo, const void* cpl, const void* mat, const void* b, void* x,
                         void* r, int ov, cudaStream_t st) {
  switch (s) {
    case 4: return gen_launch<T, V, 4>(mode, warps, nb, nbp, pos0, npos, perm, tptr, tinfo, cpl, mat, b, x, r, ov, st);
    case 9: return gen_launch<T, V, 9>(mode, warps, nb, nbp, pos0, npos, perm, tptr, tinfo, cpl, mat, b, x, r, ov, st);
    case 16: return gen_launch<T, V, 16>(mode, warps, nb, nbp, pos0, npos, perm, tptr, tinfo, cpl, mat, b, x, r, ov, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_gen_element(int storage, int mode, int warps, int s, int nb, int nbp, int pos0, int npos,
                               const int* perm, const int* tptr, const int* tinfo, const void* cpl, const void* mat,
                               const void* b, void* x, void* r, cudaStream_t st, int ov) {
  if (npos <= 0) return cudaSuccess;
  if (nb != 3 * s || nb > kGenMaxNb) return cudaErrorInvalidValue;
  // the 16-column kernels read the iterate with 16-byte loads
  if (s == 16 && (((uintptr_t)x | (uintptr_t)b) & 15)) return cudaErrorMisalignedAddress;
  if (storage == STK_FP64)
    return gen_dispatch<double, double>(mode, warps, s, nb, nbp, pos0, npos, perm, tptr, tinfo, cpl, mat, b, x, r,
                                        ov, st);
  if (storage == STK_FP32)
    return gen_dispatch<float, float>(mode, warps, s, nb, nbp, pos0, npos, perm, tptr, tinfo, cpl, mat, b, x, r, ov,
                                      st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_gen_restrict(int vec64, int nc, int s, int nb, const int* cptr, const int* clist, const void* I,
                                const void* r, void* rc, cudaStream_t st) {
  const int64_t n = (int64_t)nc * nb;
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)((n + 255) / 256);
  if (vec64)
    gen_restrict_kernel<double, double><<<blocks, 256, 0, st>>>(nc, s, nb, cptr, clist, (const double*)I,
                                                                (const double*)r, (double*)rc);
  else
    gen_restrict_kernel<float, float><<<blocks, 256, 0, st>>>(nc, s, nb, cptr, clist, (const float*)I,
                                                              (const float*)r, (float*)rc);
  return cudaGetLastError();
}

cudaError_t launch_gen_prolong(int vec64, int nf, int s, int nb, const int* parent, const void* I, const void* xc,
                               void* x, cudaStream_t st) {
  const int64_t n = (int64_t)nf * nb;
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)((n + 255) / 256);
  if (vec64)
    gen_prolong_kernel<double, double><<<blocks, 256, 0, st>>>(nf, s, nb, parent, (const double*)I,
                                                               (const double*)xc, (double*)x);
  else
    gen_prolong_kernel<float, float><<<blocks, 256, 0, st>>>(nf, s, nb, parent, (const float*)I,
                                                             (const float*)xc, (float*)x);
  return cudaGetLastError();
}

}  // namespace stk
