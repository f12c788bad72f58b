// C ABI of the Stokes multigrid library (declarations and contracts in
// include/stokes_mg.h): context management, device packing of the hierarchy
// built by setup.cpp, and the host drivers of the V-cycle (Algorithm 1 of
// arXiv:1911.05888) and of the outer iteration.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "stk_internal.h"
#include "../../include/stokes_mg.h"


using namespace stk;

namespace stk {

// One element-kernel launch (colour step or residual) on level l: launches of
// few elements (npos <= wide_max) take the one-CTA-per-element latency
// variant, the others the configured variant; the pipelined variant falls
// back to direct loads when its records do not fit in shared memory.
cudaError_t run_element(Ctx& c, int l, int prec, int mode, int pos0, int npos, const void* mat, const void* b,
                        void* x, void* r, cudaStream_t st) {
  return run_element_on(c, c.pat, c.dev[l], prec, mode, pos0, npos, mat, b, x, r, st);
}

// The same on any level's records with its own pattern (the cluster level's).
cudaError_t run_element_on(Ctx& c, const Pattern& pat, DevLevel& D, int prec, int mode, int pos0, int npos,
                           const void* mat, const void* b, void* x, void* r, cudaStream_t st) {
  if (D.gen)   // general block-sparse level (cut-cell hierarchy)
    return launch_gen_element(prec, mode, c.gen_warps, c.s, c.nb, D.nbp, pos0, npos, D.perm, D.tptr, D.tinfo,
                              D.cpl[prec], mat, b, x, r, st, c.launch_overlap);
  // FP16 records carry scales and run on the warp and wide kernels only.
  const bool scaled = prec == STK_FP16;
  const float* tsc = scaled ? D.csc : nullptr;
  const float* rsc = scaled ? (mode == MODE_GS ? D.isc : D.dsc) : nullptr;
  if (npos <= c.wide_max) {
    cudaError_t e = launch_element_wide(pat, prec, mode, pos0, npos, D.perm, D.nbr, D.cpl[prec], mat, tsc, rsc, b,
                                        x, r, st, c.launch_overlap);
    if (e != cudaErrorInvalidValue || scaled) return e;
  }
  const int variant = c.variant_of[prec];
  if (variant == 3) {   // 16-bit records, next element staged while this one computes
    cudaError_t e = launch_element_ring(pat, prec, c.ring_warps[prec], mode, pos0, npos, D.perm, D.nbr, D.cpl[prec],
                                        mat, tsc, rsc, b, x, r, c.launch_overlap, st);
    if (e != cudaErrorInvalidValue) return e;
  }
  if (variant >= 2 || scaled) {
    cudaError_t e = launch_element_warp(pat, prec, mode, pos0, npos, D.perm, D.nbr, D.cpl[prec], mat, tsc, rsc, b,
                                        x, r, c.warp_ctas[prec], st, c.launch_overlap);
    if (e != cudaErrorInvalidValue || scaled) return e;
  }
  if (variant == 1) {
    cudaError_t e = launch_element_pipe(pat, prec, mode, pos0, npos, D.perm, D.nbr, D.cpl[prec], mat, b, x, r,
                                        c.dev_err, c.pipe_ctas[prec], c.pipe_stages[prec], st);
    if (e != cudaErrorInvalidValue) return e;
  }
  return launch_element(pat, prec, mode, pos0, npos, D.perm, D.nbr, D.cpl[prec], mat, b, x, r, st);
}

}  // namespace stk

namespace {

void free_persist(Ctx& c);
int persist_grid(const Ctx& c);
void build_persist(Ctx& c);


struct CudaFail {
  cudaError_t e;
  const char* what;
};

inline void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw CudaFail{e, what};
}

template <typename F>
int guard(stk_ctx* c, F&& fn) {
  if (!c) return STK_ERR_INVALID_ARG;
  try {
    c->err.clear();
    return fn();
  } catch (const CudaFail& f) {
    c->err = std::string(f.what) + ": " + cudaGetErrorString(f.e);
    return STK_ERR_CUDA;
  } catch (const std::bad_alloc&) {
    c->err = "host allocation failed";
    return STK_ERR_OOM;
  } catch (...) {
    c->err = "unexpected internal error";
    return STK_ERR_INVALID_ARG;
  }
}

int fail(stk_ctx* c, int code, const std::string& msg) {
  c->err = msg;
  return code;
}

void* dalloc(Ctx& c, size_t bytes) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
  if (e != cudaSuccess) throw CudaFail{e, "cudaMalloc"};
  c.allocations.push_back(p);
  c.device_bytes += (int64_t)(bytes ? bytes : 16);
  return p;
}

void free_device(Ctx& c) {
  for (void* p : c.allocations) cudaFree(p);
  c.allocations.clear();
  c.device_bytes = 0;
  free_persist(c);
  c.gbar = nullptr;
  c.cluster_on = 0;
  c.cdev = DevLevel();
  c.chost = HostLevel();
  for (int v = 0; v < 2; ++v) c.cvx[v] = c.cvb[v] = c.cvr[v] = c.ctmp[v] = nullptr;
  if (c.norm_host) cudaFreeHost(c.norm_host);
  c.norm_host = nullptr;
  if (c.khost) cudaFreeHost(c.khost);
  c.khost = nullptr;
  if (c.mkhost) cudaFreeHost(c.mkhost);
  c.mkhost = nullptr;
  c.mkV = c.mkZ = c.mkw = c.mkzero = c.mkpart = c.mkdev = nullptr;
  c.mkz32 = c.mkw32 = c.mkzero32 = nullptr;
  c.mk_cap = c.mk_nr = 0;
  c.kV = c.kZ = c.kw = c.kzero = c.kpart = c.kdots = nullptr;
  c.kcap = 0;
  if (c.cycle_graph) cudaGraphExecDestroy(c.cycle_graph);
  c.cycle_graph = nullptr;
  c.cycle_graph_prec = -1;
  if (c.mgraph) cudaGraphExecDestroy(c.mgraph);
  c.mgraph = nullptr;
  c.mgraph_key[0] = c.mgraph_key[1] = c.mgraph_key[2] = -1;
  c.mr_nr = 0;
  c.mX = c.mB = c.mR = c.mNorm = c.mPart = nullptr;
  c.mRin = c.mRb = c.mAcc = nullptr;
  if (c.graph) cudaGraphExecDestroy(c.graph);
  c.graph = nullptr;
  c.graph_x = c.graph_b = nullptr;
  if (c.lgraph) cudaGraphExecDestroy(c.lgraph);
  if (c.rgraph) cudaGraphExecDestroy(c.rgraph);
  c.lgraph = c.rgraph = nullptr;
  c.lgraph_x = c.lgraph_b = nullptr;
  c.dev.clear();
  c.ready = false;
}

int64_t level_ne(const Ctx& c, int l) { return c.host[l].ne; }
int nlevels(const Ctx& c) { return (int)c.host.size(); }

// Colouring of a single-phase level: the checkerboard (i_1 + ... + i_d) mod 2
// when the operator couples face neighbours only (standard form), else the
// 2^d parity colouring sum_k (i_k mod 2) 2^k, which also separates the
// diagonal / edge couplings of the viscous-stress form (Section 3 asks only
// for a valid multi-colouring).
bool checkerboard(const Ctx& c) {
  return c.colouring == STK_COLOURS_CHECKERBOARD || (c.colouring == STK_COLOURS_AUTO && c.gamma == 0);
}

int colour_of(const Ctx& c, const int* n, int64_t e) {
  int idx[3];
  element_index(n, c.d, e, idx);
  int col = 0;
  if (checkerboard(c)) {
    for (int k = 0; k < c.d; ++k) col += idx[k];
    return col & 1;
  }
  for (int k = 0; k < c.d; ++k) col |= (idx[k] & 1) << k;
  return col;
}

// Pack the Stokes blocks of smoothing level l into the colour-major device
// records of kernels.cu.
void pack_records(Ctx& c, const HostLevel& H, const Pattern& P, DevLevel& D, bool level0, cudaStream_t st) {
  int s = P.s, nb = P.nb, ss = s * s;
  int64_t ne = H.ne;
  D.ne = (int)ne;
  for (int k = 0; k < 3; ++k) D.n[k] = H.n[k];
  // Parity colouring (single phase) or greedy colouring (phases: the
  // interphase lifts couple elements two apart along an axis).
  std::vector<int> colour(ne);
  if (!H.chi.empty())
    greedy_colours(c, H.n, colour);
  else
    for (int64_t e = 0; e < ne; ++e) colour[e] = colour_of(c, H.n, e);
  int ncol = 0;
  for (int v : colour) ncol = std::max(ncol, v + 1);
  if (ncol > 64) throw std::runtime_error("more than 64 colours");
  D.ncolour = ncol;
  std::vector<int> perm;
  perm.reserve(ne);
  D.cstart[0] = 0;
  for (int col = 0; col < ncol; ++col) {
    for (int64_t e = 0; e < ne; ++e)
      if (colour[e] == col) perm.push_back((int)e);
    D.cstart[col + 1] = (int)perm.size();
  }
  std::vector<int> nbr((size_t)ne * P.NO);
  for (int64_t pos = 0; pos < ne; ++pos)
    for (int o = 0; o < P.NO; ++o) nbr[(size_t)pos * P.NO + o] = H.nbr[(size_t)perm[pos] * P.NO + o];
  D.perm = (int*)dalloc(c, ne * sizeof(int));
  D.nbr = (int*)dalloc(c, nbr.size() * sizeof(int));
  ck(cudaMemcpy(D.perm, perm.data(), ne * sizeof(int), cudaMemcpyHostToDevice), "copy perm");
  ck(cudaMemcpy(D.nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice), "copy nbr");

  // Inverses of the diagonal blocks (FP64, host).
  std::vector<double> Dinv((size_t)ne * nb * nb);
  std::string err;
  int rc = invert_blocks(nb, (int)ne, H.D.data(), Dinv.data(), err);
  if (rc != STK_OK) throw std::runtime_error(err);

  size_t cpl_n = (size_t)ne * s * P.TRP, mat_n = (size_t)ne * nb * P.NBP;
  std::vector<double> buf(std::max(cpl_n, mat_n));
  // couplings: rec[c][tr], tr = t*s + i holds C[t][i][c]
  std::fill(buf.begin(), buf.begin() + cpl_n, 0.0);
  for (int64_t pos = 0; pos < ne; ++pos) {
    int64_t e = perm[pos];
    double* rec = &buf[(size_t)pos * s * P.TRP];
    for (int t = 0; t < P.T; ++t)
      for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j)
          rec[(size_t)j * P.TRP + t * s + i] = H.C[((size_t)e * P.T + t) * ss + i * s + j];
  }
  D.cpl[0] = dalloc(c, cpl_n * sizeof(double));
  ck(cudaMemcpy(D.cpl[0], buf.data(), cpl_n * sizeof(double), cudaMemcpyHostToDevice), "copy cpl");
  auto pack_mat = [&](const std::vector<double>& M, void*& out) {
    std::fill(buf.begin(), buf.begin() + mat_n, 0.0);
    for (int64_t pos = 0; pos < ne; ++pos) {
      int64_t e = perm[pos];
      double* rec = &buf[(size_t)pos * nb * P.NBP];
      const double* m = &M[(size_t)e * nb * nb];
      for (int r = 0; r < nb; ++r)
        for (int cc = 0; cc < nb; ++cc) rec[(size_t)cc * P.NBP + r] = m[(size_t)r * nb + cc];
    }
    out = dalloc(c, mat_n * sizeof(double));
    ck(cudaMemcpy(out, buf.data(), mat_n * sizeof(double), cudaMemcpyHostToDevice), "copy mat");
  };
  pack_mat(Dinv, D.inv[0]);
  pack_mat(H.D, D.dia[0]);
  // Low-precision copies (rounded once from FP64: round to nearest even).
  if (c.precision == STK_FP32 || c.precision == STK_BF16) {
    int pr = c.precision;
    size_t es = (pr == STK_FP32) ? 4 : 2;
    void* src[3] = {D.cpl[0], D.inv[0], D.dia[0]};
    size_t cnt[3] = {cpl_n, mat_n, mat_n};
    void** dst[3] = {&D.cpl[pr], &D.inv[pr], &D.dia[pr]};
    for (int i = 0; i < 3; ++i) {
      *dst[i] = dalloc(c, cnt[i] * es);
      if (pr == STK_FP32)
        ck(launch_convert(0, 1, (int64_t)cnt[i], *dst[i], src[i], st), "convert fp32");
      else
        ck(launch_to_bf16((int64_t)cnt[i], *dst[i], (const double*)src[i], st), "convert bf16");
    }
  }
  // FP16 copies with power-of-two scales per coupling sub-block and per row
  // of the dense blocks.
  if (c.precision == STK_FP16) {
    const int TP = (P.T + 3) / 4 * 4;
    D.cpl[STK_FP16] = dalloc(c, cpl_n * 2);
    D.csc = (float*)dalloc(c, (size_t)ne * TP * sizeof(float));
    ck(launch_to_fp16_tasks(ne, s, P.T, P.TRP, D.cpl[STK_FP16], D.csc, (const double*)D.cpl[0], st),
       "convert fp16 couplings");
    D.inv[STK_FP16] = dalloc(c, mat_n * 2);
    D.isc = (float*)dalloc(c, (size_t)ne * P.NBP * sizeof(float));
    ck(launch_to_fp16_rows(ne, nb, P.NBP, D.inv[STK_FP16], D.isc, (const double*)D.inv[0], st), "convert fp16 inv");
    D.dia[STK_FP16] = dalloc(c, mat_n * 2);
    D.dsc = (float*)dalloc(c, (size_t)ne * P.NBP * sizeof(float));
    ck(launch_to_fp16_rows(ne, nb, P.NBP, D.dia[STK_FP16], D.dsc, (const double*)D.dia[0], st), "convert fp16 dia");
  }
  // With 16-bit smoother records the refined Krylov matvec still runs on FP32
  // couplings and diagonal blocks: its Arnoldi relation needs u * cond(A) < 1,
  // which 16-bit unit roundoffs (2^-8, 2^-11) do not give on these operators.
  if (level0 && (c.precision == STK_BF16 || c.precision == STK_FP16)) {
    void* src[2] = {D.cpl[0], D.dia[0]};
    size_t cnt[2] = {cpl_n, mat_n};
    void** dst[2] = {&D.cpl[STK_FP32], &D.dia[STK_FP32]};
    for (int i = 0; i < 2; ++i) {
      *dst[i] = dalloc(c, cnt[i] * 4);
      ck(launch_convert(0, 1, (int64_t)cnt[i], *dst[i], src[i], st), "convert fp32");
    }
  }
  // FP32 remainders for the FP64-accurate FGMRES matvec on the FP32 units
  if (level0 && c.precision != STK_FP64) {
    D.cpl_lo = dalloc(c, cpl_n * 4);
    D.dia_lo = dalloc(c, mat_n * 4);
    ck(launch_fp32_remainder((int64_t)cpl_n, (const double*)D.cpl[0], D.cpl_lo, st), "remainder");
    ck(launch_fp32_remainder((int64_t)mat_n, (const double*)D.dia[0], D.dia_lo, st), "remainder");
  }
  (void)st;
}

void pack_level(Ctx& c, int l, cudaStream_t st) { pack_records(c, c.host[l], c.pat, c.dev[l], l == 0, st); }

// Device records of a general block-sparse level (cut-cell hierarchy): the
// colour-major element order, every position's task range and task words,
// the coupling records [task][s][s] row-major, A_ii^{-1} and A_ii
// column-major [pos][nb][nb], and the injection to the next coarser level.
void pack_generic(Ctx& c, int l, cudaStream_t st) {
  const HostLevel& H = c.host[l];
  DevLevel& D = c.dev[l];
  const int s = c.s, nb = c.nb, ss = s * s, ne = H.ne;
  D.gen = 1;
  D.ne = ne;
  D.nbp = (nb + 3) / 4 * 4;   // columns of 16-byte multiples in FP32 and FP64 (cp.async staging)
  for (int k = 0; k < 3; ++k) D.n[k] = H.n[k];
  int ncol = 0;
  for (int v : H.colour) ncol = std::max(ncol, v + 1);
  if (ncol > 64) throw std::runtime_error("more than 64 colours");
  D.ncolour = ncol;
  std::vector<int> perm;
  perm.reserve(ne);
  D.cstart[0] = 0;
  for (int col = 0; col < ncol; ++col) {
    for (int e = 0; e < ne; ++e)
      if (H.colour[e] == col) perm.push_back(e);
    D.cstart[col + 1] = (int)perm.size();
  }
  std::vector<int> tptr(ne + 1, 0), tinfo;
  std::vector<double> rec;
  rec.reserve(H.C.size());
  for (int pos = 0; pos < ne; ++pos) {
    const int e = perm[pos];
    for (int t = H.tptr[e]; t < H.tptr[e + 1]; ++t) {
      tinfo.push_back(H.tnbr[t] * 16 + (H.tvar[t] / 4) * 4 + H.tvar[t] % 4);
      rec.insert(rec.end(), H.C.begin() + (size_t)t * ss, H.C.begin() + (size_t)(t + 1) * ss);
    }
    tptr[pos + 1] = (int)tinfo.size();
  }
  if ((int64_t)ne * 16 >= (int64_t)1 << 31) throw std::runtime_error("too many elements for the task words");
  D.perm = (int*)dalloc(c, (size_t)ne * sizeof(int));
  D.tptr = (int*)dalloc(c, tptr.size() * sizeof(int));
  D.tinfo = (int*)dalloc(c, std::max<size_t>(1, tinfo.size()) * sizeof(int));
  ck(cudaMemcpy(D.perm, perm.data(), (size_t)ne * sizeof(int), cudaMemcpyHostToDevice), "copy perm");
  ck(cudaMemcpy(D.tptr, tptr.data(), tptr.size() * sizeof(int), cudaMemcpyHostToDevice), "copy tptr");
  if (!tinfo.empty())
    ck(cudaMemcpy(D.tinfo, tinfo.data(), tinfo.size() * sizeof(int), cudaMemcpyHostToDevice), "copy tinfo");
  D.cpl[0] = dalloc(c, std::max<size_t>(1, rec.size()) * sizeof(double));
  if (!rec.empty())
    ck(cudaMemcpy(D.cpl[0], rec.data(), rec.size() * sizeof(double), cudaMemcpyHostToDevice), "copy cpl");
  std::vector<double> Dinv((size_t)ne * nb * nb);
  std::string err;
  if (invert_blocks(nb, ne, H.D.data(), Dinv.data(), err) != STK_OK) throw std::runtime_error(err);
  const int nbp = D.nbp;
  const size_t mat_n = (size_t)ne * nb * nbp;
  std::vector<double> buf(mat_n, 0.0);
  auto pack_mat = [&](const std::vector<double>& M, void*& out) {
    for (int pos = 0; pos < ne; ++pos) {
      const double* m = &M[(size_t)perm[pos] * nb * nb];
      double* o = &buf[(size_t)pos * nb * nbp];
      for (int r = 0; r < nb; ++r)
        for (int cc = 0; cc < nb; ++cc) o[(size_t)cc * nbp + r] = m[(size_t)r * nb + cc];
    }
    out = dalloc(c, mat_n * sizeof(double));
    ck(cudaMemcpy(out, buf.data(), mat_n * sizeof(double), cudaMemcpyHostToDevice), "copy mat");
  };
  pack_mat(Dinv, D.inv[0]);
  pack_mat(H.D, D.dia[0]);
  if (c.precision == STK_FP32) {
    void* src[3] = {D.cpl[0], D.inv[0], D.dia[0]};
    size_t cnt[3] = {std::max<size_t>(1, rec.size()), mat_n, mat_n};
    void** dst[3] = {&D.cpl[1], &D.inv[1], &D.dia[1]};
    for (int i = 0; i < 3; ++i) {
      *dst[i] = dalloc(c, cnt[i] * 4);
      ck(launch_convert(0, 1, (int64_t)cnt[i], *dst[i], src[i], st), "convert fp32");
    }
  }
  // injection to the next coarser level
  if (!H.parent.empty()) {
    const int nc = c.host[l + 1].ne;
    std::vector<int> cptr(nc + 1, 0), clist(ne);
    for (int f = 0; f < ne; ++f) cptr[H.parent[f] + 1]++;
    for (int k = 0; k < nc; ++k) cptr[k + 1] += cptr[k];
    std::vector<int> fill(cptr.begin(), cptr.end() - 1);
    for (int f = 0; f < ne; ++f) clist[fill[H.parent[f]]++] = f;
    D.gparent = (int*)dalloc(c, (size_t)ne * sizeof(int));
    D.gcptr = (int*)dalloc(c, cptr.size() * sizeof(int));
    D.gclist = (int*)dalloc(c, clist.size() * sizeof(int));
    ck(cudaMemcpy(D.gparent, H.parent.data(), (size_t)ne * sizeof(int), cudaMemcpyHostToDevice), "copy parent");
    ck(cudaMemcpy(D.gcptr, cptr.data(), cptr.size() * sizeof(int), cudaMemcpyHostToDevice), "copy cptr");
    ck(cudaMemcpy(D.gclist, clist.data(), clist.size() * sizeof(int), cudaMemcpyHostToDevice), "copy clist");
    D.gI[0] = dalloc(c, H.Ib.size() * sizeof(double));
    ck(cudaMemcpy(D.gI[0], H.Ib.data(), H.Ib.size() * sizeof(double), cudaMemcpyHostToDevice), "copy injection");
    D.gI[1] = dalloc(c, H.Ib.size() * sizeof(float));
    ck(launch_convert(0, 1, (int64_t)H.Ib.size(), D.gI[1], D.gI[0], st), "convert injection");
  }
}


void alloc_vectors(Ctx& c) {
  int L = nlevels(c);
  for (int l = 0; l < L; ++l) {
    DevLevel& D = c.dev[l];
    int64_t n = level_ne(c, l) * c.nb;
    D.ne = (int)level_ne(c, l);
    for (int k = 0; k < 3; ++k) D.n[k] = c.host[l].n[k];
    for (int v = 0; v < 2; ++v) {
      if (v == 1 && c.precision == STK_FP64) continue;
      size_t es = v == 0 ? 8 : 4;
      D.vx[v] = dalloc(c, n * es);
      D.vb[v] = dalloc(c, n * es);
      D.vr[v] = dalloc(c, n * es);
    }
  }
  int64_t n0 = level_ne(c, 0) * c.nb;
  c.r64 = (double*)dalloc(c, n0 * 8);
  c.c64 = (double*)dalloc(c, n0 * 8);
  c.norm_buf = (double*)dalloc(c, 1104 * 8);   // scalars, 1024 partials, probe slots
  ck(cudaMallocHost(&c.norm_host, 8 * sizeof(double)), "cudaMallocHost");
}

// ---- large bottom levels: eigendecomposition by cuSOLVER (loaded at run time)
// The same steps as the host solver for 301-1200 unknowns (stk_host_pseudo_inverse):
// equilibrate A^ = S A S (S_i = row 1-norm^(-1/2)), eigendecompose A^ (here on
// the device), snap |lambda| <= theta max|lambda|, G = S A^+ S, then project G
// off the kernel of A (the vectors S v_k of the snapped eigenvalues).
// pinv(i, j) = S_i S_j sum_k V(i, k) w_k V(j, k), V column-major (n x n),
// w = 1/lambda or 0.
__global__ void pinv_gemm_kernel(int n, const double* __restrict__ V, const double* __restrict__ w,
                                 const double* __restrict__ S, double* __restrict__ P) {
  __shared__ double As[16][17], Bs[16][17];
  const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
  double acc = 0.0;
  for (int k0 = 0; k0 < n; k0 += 16) {
    const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
    const int ib = blockIdx.x * 16 + threadIdx.x;
    As[threadIdx.y][threadIdx.x] = (i < n && ka < n) ? V[(size_t)ka * n + i] * w[ka] : 0.0;
    Bs[threadIdx.y][threadIdx.x] = (ib < n && kb < n) ? V[(size_t)kb * n + ib] : 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc += As[threadIdx.y][k] * Bs[k][threadIdx.x];
    __syncthreads();
  }
  if (i < n && j < n) P[(size_t)i * n + j] = S[i] * S[j] * acc;
}

typedef int (*syevd_buf_fn)(void*, int, int, int, const double*, int, const double*, int*);
typedef int (*syevd_fn)(void*, int, int, int, double*, int, double*, double*, int, int*);
typedef int (*create_fn)(void**);
typedef int (*destroy_fn)(void*);

// Owns what the cuSOLVER path acquires; releases all of it on every return.
struct CusolverScope {
  void* so = nullptr;
  void* handle = nullptr;
  destroy_fn destroy = nullptr;
  std::vector<void*> dev;
  ~CusolverScope() {
    for (void* p : dev) cudaFree(p);
    if (handle && destroy) destroy(handle);
    if (so) dlclose(so);
  }
  bool alloc(void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) return false;
    dev.push_back(*p);
    return true;
  }
};

// Returns false when cuSOLVER cannot be loaded or fails (the caller then uses
// the host solver).
bool pseudo_inverse_cusolver(Ctx& c, int n, const std::vector<double>& A, double* d_pinv, int& snapped,
                             double theta) {
  CusolverScope g;
  for (const char* name : {"libcusolver.so", "libcusolver.so.12", "libcusolver.so.11"})
    if ((g.so = dlopen(name, RTLD_NOW | RTLD_LOCAL))) break;
  if (!g.so) return false;
  auto create = (create_fn)dlsym(g.so, "cusolverDnCreate");
  g.destroy = (destroy_fn)dlsym(g.so, "cusolverDnDestroy");
  auto bufsz = (syevd_buf_fn)dlsym(g.so, "cusolverDnDsyevd_bufferSize");
  auto syevd = (syevd_fn)dlsym(g.so, "cusolverDnDsyevd");
  if (!create || !g.destroy || !bufsz || !syevd) return false;
  if (create(&g.handle) != 0) {
    g.handle = nullptr;
    return false;
  }
  const int JOBZ_VECTOR = 1, FILL_LOWER = 0;   // CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER
  std::vector<double> S, Ah;
  equilibrate_sym(n, A, S, Ah);
  double *dA = nullptr, *dW = nullptr, *dWork = nullptr, *dInv = nullptr, *dS = nullptr;
  int* dInfo = nullptr;
  int lwork = 0, info = 1;
  std::vector<double> lam(n), inv(n, 0.0);
  if (!g.alloc((void**)&dA, (size_t)n * n * 8) || !g.alloc((void**)&dW, (size_t)n * 8) ||
      !g.alloc((void**)&dInv, (size_t)n * 8) || !g.alloc((void**)&dS, (size_t)n * 8) ||
      !g.alloc((void**)&dInfo, sizeof(int)))
    return false;
  // A^ is symmetric: row-major and column-major storage coincide.
  if (cudaMemcpy(dA, Ah.data(), (size_t)n * n * 8, cudaMemcpyHostToDevice) != cudaSuccess) return false;
  if (cudaMemcpy(dS, S.data(), (size_t)n * 8, cudaMemcpyHostToDevice) != cudaSuccess) return false;
  if (bufsz(g.handle, JOBZ_VECTOR, FILL_LOWER, n, dA, n, dW, &lwork) != 0) return false;
  if (!g.alloc((void**)&dWork, (size_t)std::max(lwork, 1) * 8)) return false;
  if (syevd(g.handle, JOBZ_VECTOR, FILL_LOWER, n, dA, n, dW, dWork, lwork, dInfo) != 0) return false;
  if (cudaMemcpy(&info, dInfo, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || info != 0) return false;
  if (cudaMemcpy(lam.data(), dW, (size_t)n * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
  std::vector<int> kern;
  double lmax = 0.0;
  for (double l : lam) lmax = std::max(lmax, std::fabs(l));
  for (int k = 0; k < n; ++k) {
    if (std::fabs(lam[k]) <= theta * lmax) kern.push_back(k);
    else inv[k] = 1.0 / lam[k];
  }
  if (cudaMemcpy(dInv, inv.data(), (size_t)n * 8, cudaMemcpyHostToDevice) != cudaSuccess) return false;
  dim3 blk(16, 16), grd((n + 15) / 16, (n + 15) / 16);
  pinv_gemm_kernel<<<grd, blk>>>(n, dA, dInv, dS, d_pinv);
  c.launches++;
  if (cudaDeviceSynchronize() != cudaSuccess) return false;
  const int nk = (int)kern.size();
  if (nk > 0) {
    // kernel vectors of A: S v_k (column kern[a] of the column-major V)
    std::vector<double> K((size_t)nk * n), G((size_t)n * n);
    for (int a = 0; a < nk; ++a)
      if (cudaMemcpy(&K[(size_t)a * n], dA + (size_t)kern[a] * n, (size_t)n * 8, cudaMemcpyDeviceToHost) !=
          cudaSuccess)
        return false;
    for (int a = 0; a < nk; ++a)
      for (int j = 0; j < n; ++j) K[(size_t)a * n + j] *= S[j];
    if (cudaMemcpy(G.data(), d_pinv, (size_t)n * n * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    project_off_kernel(n, G, K, nk);
    if (cudaMemcpy(d_pinv, G.data(), (size_t)n * n * 8, cudaMemcpyHostToDevice) != cudaSuccess) return false;
  }
  snapped = nk;
  return true;
}

// Bottom level: dense operator, eigen pseudo-inverse, to device.
void setup_bottom(Ctx& c) {
  const HostLevel& H = c.host.back();
  const Pattern& P = c.pat;
  int nb = c.nb, s = c.s, ss = s * s;
  int64_t ne = H.ne, n = ne * nb;
  std::vector<double> A((size_t)n * n, 0.0);
  for (int64_t a = 0; a < ne; ++a) {
    for (int r = 0; r < nb; ++r)
      for (int cc = 0; cc < nb; ++cc)
        A[(size_t)(a * nb + r) * n + a * nb + cc] += H.D[(size_t)a * nb * nb + r * nb + cc];
    if (c.cut) {
      // general block-sparse level: the element's coupling tasks
      for (int t = H.tptr[a]; t < H.tptr[a + 1]; ++t) {
        const int64_t bb = H.tnbr[t];
        const int rv = H.tvar[t] / 4, cv = H.tvar[t] % 4;
        for (int i = 0; i < s; ++i)
          for (int j = 0; j < s; ++j)
            A[(size_t)(a * nb + rv * s + i) * n + bb * nb + cv * s + j] += H.C[(size_t)t * ss + i * s + j];
      }
      continue;
    }
    for (int t = 0; t < P.T; ++t) {
      int64_t bb = H.nbr[(size_t)a * P.NO + P.task_o[t]];
      if (bb < 0) continue;
      int rv = P.task_rv[t], cv = P.task_cv[t];
      for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j)
          A[(size_t)(a * nb + rv * s + i) * n + bb * nb + cv * s + j] +=
              H.C[((size_t)a * P.T + t) * ss + i * s + j];
    }
  }
  c.nbot = n;
  c.bottom_pinv = (double*)dalloc(c, (size_t)n * n * sizeof(double));
  // Cyclic Jacobi (O(n^3) per sweep, under a second up to 300 unknowns) for
  // small bottom levels; the equilibrated Householder-QR solver up to 1200
  // (a 864-unknown 3D bottom: 0.8 s instead of 30-90 s); cuSOLVER's symmetric
  // eigensolver above.
  if (n > 1200 && pseudo_inverse_cusolver(c, (int)n, A, c.bottom_pinv, c.n_snapped, 1e-10)) {
    c.bottom_solver = 2;
    return;
  }
  std::vector<double> pinv;
  c.bottom_solver = n <= 300 ? 0 : 1;
  const int rc = n <= 300 ? pseudo_inverse_jacobi((int)n, A, pinv, c.n_snapped, 1e-10)
                          : pseudo_inverse_sym((int)n, A, pinv, c.n_snapped, 1e-10);
  if (rc != STK_OK) throw std::runtime_error("bottom solver");
  ck(cudaMemcpy(c.bottom_pinv, pinv.data(), (size_t)n * n * sizeof(double), cudaMemcpyHostToDevice),
     "copy bottom");
}

// ---- learned post-smoother on the finest level -------------------------------------
// delta (into c.lxt) from the cycle's own residual after its post-smoothing:
// r_c = b_c - A x_c with the cycle's records (FP32 vectors), features of r_c,
// the two layers, delta_i = ||r_c,i|| y_i.
void enqueue_learned_delta(Ctx& c, int prec, const void* xv, const void* bv, cudaStream_t st) {
  DevLevel& D0 = c.dev[0];
  const int ne = D0.ne, nb = c.nb, nface = 2 * c.d;
  ck(run_element(c, 0, prec, MODE_RESID, 0, ne, D0.dia[prec], bv, (void*)xv, D0.vr[1], st), "learned residual");
  ck(launch_features(ne, nb, nface, c.l_no, c.l_ldf, c.l_nbr, (const float*)D0.vr[1], c.lF, c.lnrm, st), "features");
  ck(launch_sgemm(ne, c.l_hid, c.l_in, 0, 0, c.lF, c.l_ldf, c.lW1, c.l_hid, c.lH, c.l_hid, c.lb1, 1, 1.f, 0.f, st),
     "layer 1");
  ck(launch_sgemm(ne, nb, c.l_hid, 0, 0, c.lH, c.l_hid, c.lW2, nb, c.lY, nb, c.lb2, 0, 1.f, 0.f, st), "layer 2");
  ck(launch_apply_correction(ne, nb, nb, c.l_zero, c.lnrm, c.lY, c.lxt, st), "delta");
  c.launches += 5;
}

// ---- the V-cycle (Algorithm 1) ------------------------------------------------
// Smoothing sweeps of one phase on level l: nu * growth^l, but no more than
// max(nu, cap).  growth 1 keeps Algorithm 1's fixed counts; growth 2 is the
// variable V-cycle named in Section 6 (more smoothing on coarser levels).
int level_sweeps(const Ctx& c, int nu, int l) {
  int64_t s = nu;
  const int64_t cap = std::max<int64_t>(nu, c.cyc_cap);
  for (int k = 0; k < l && s < cap; ++k) s *= c.cyc_growth;
  return (int)std::min(s, cap);
}

// Visits to level l+1 per visit of level l: gamma (1 = V-cycle, 2 = W-cycle,
// Section 6), except that the coarsest level, solved exactly, is visited once.
int coarse_visits(const Ctx& c, int l) { return l + 1 == nlevels(c) - 1 ? 1 : c.cyc_gamma; }

// prec: storage precision of the blocks; vectors FP64 when prec == 0, else FP32.
void enqueue_smooth(Ctx& c, int prec, int l, int sweeps, void* x, const void* b, cudaStream_t st) {
  DevLevel& D = c.dev[l];
  for (int it = 0; it < sweeps; ++it)
    for (int col = 0; col < D.ncolour; ++col) {
      int n = D.cstart[col + 1] - D.cstart[col];
      if (n <= 0) continue;
      ck(run_element(c, l, prec, MODE_GS, D.cstart[col], n, D.inv[prec], b, x, nullptr, st), "gs colour launch");
      c.launches++;
    }
}

void enqueue_cycle_clustered(Ctx& c, int prec, void* x, const void* b, cudaStream_t st);

void enqueue_cycle(Ctx& c, int prec, int l, void* x, const void* b, cudaStream_t st) {
  int vi = prec == STK_FP64 ? 0 : 1;
  int L = nlevels(c);
  if (l == 0 && c.cluster_on) {
    enqueue_cycle_clustered(c, prec, x, b, st);
    return;
  }
  if (l >= 1 && l == c.persist_level[prec] && c.persist_prog[prec] && x == c.dev[l].vx[vi] &&
      b == c.dev[l].vb[vi]) {
    // levels l .. L-1 in one cooperative launch (persist.cu)
    ck(cudaMemsetAsync(c.gbar, 0, sizeof(GridBarrierWords), st), "barrier reset");
    ck(launch_coarse_cycle(c.pat, prec, c.persist_prog[prec], c.persist_nphase[prec], c.gbar, c.dev_err,
                           c.barrier_limit, persist_grid(c), st),
       "persistent coarse cycle");
    c.launches++;
    return;
  }
  if (l == L - 1) {
    ck(launch_bottom(vi == 0, c.nbot, c.bottom_pinv, b, x, st), "bottom launch");
    c.launches++;
    return;
  }
  DevLevel& D = c.dev[l];
  DevLevel& Dc = c.dev[l + 1];
  enqueue_smooth(c, prec, l, level_sweeps(c, c.nu1, l), x, b, st);
  ck(run_element(c, l, prec, MODE_RESID, 0, D.ne, D.dia[prec], b, x, D.vr[vi], st), "residual launch");
  ck(D.gen ? launch_gen_restrict(vi == 0, Dc.ne, c.s, c.nb, D.gcptr, D.gclist, D.gI[vi], D.vr[vi], Dc.vb[vi], st)
           : launch_restrict(vi == 0, c.d, c.s, c.nb, Dc.n, D.n, Dc.ne, c.child_P[vi], D.vr[vi], Dc.vb[vi], st),
     "restrict launch");
  ck(cudaMemsetAsync(Dc.vx[vi], 0, (size_t)Dc.ne * c.nb * (vi == 0 ? 8 : 4), st), "memset");
  c.launches += 2;  // residual + restriction
  for (int v = coarse_visits(c, l); v > 0; --v) enqueue_cycle(c, prec, l + 1, Dc.vx[vi], Dc.vb[vi], st);
  ck(D.gen ? launch_gen_prolong(vi == 0, D.ne, c.s, c.nb, D.gparent, D.gI[vi], Dc.vx[vi], x, st)
           : launch_prolong(vi == 0, c.d, c.s, c.nb, D.n, Dc.n, Dc.ne, c.child_PT[vi], Dc.vx[vi], x, st),
     "prolong launch");
  c.launches++;
  enqueue_smooth(c, prec, l, level_sweeps(c, c.nu2, l), x, b, st);
}

// ---- persistent coarse cycle: the phase program -------------------------------
int persist_grid(const Ctx& c) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device);
  return std::max(1, sms * c.persist_ctas);
}

// The phases enqueue_cycle would launch from level l down, in the same order.
void emit_cycle_phases(Ctx& c, int prec, int l, std::vector<CyclePhase>& prog) {
  const int vi = prec == STK_FP64 ? 0 : 1;
  const int L = nlevels(c);
  DevLevel& D = c.dev[l];
  const bool scaled = prec == STK_FP16;
  if (l == L - 1) {
    CyclePhase ph{};
    ph.op = PHASE_BOTTOM;
    ph.n = c.nbot;
    ph.tr = c.bottom_pinv;
    ph.in = D.vb[vi];
    ph.out = D.vx[vi];
    prog.push_back(ph);
    return;
  }
  DevLevel& Dc = c.dev[l + 1];
  auto smooth = [&](int sweeps) {
    for (int it = 0; it < sweeps; ++it)
      for (int col = 0; col < D.ncolour; ++col) {
        const int n = D.cstart[col + 1] - D.cstart[col];
        if (n <= 0) continue;
        CyclePhase ph{};
        ph.op = PHASE_GS;
        ph.pos0 = D.cstart[col];
        ph.n = n;
        ph.cpl = D.cpl[prec];
        ph.mat = D.inv[prec];
        ph.perm = D.perm;
        ph.nbr = D.nbr;
        ph.tsc = scaled ? D.csc : nullptr;
        ph.rsc = scaled ? D.isc : nullptr;
        ph.b = D.vb[vi];
        ph.x = D.vx[vi];
        prog.push_back(ph);
      }
  };
  smooth(level_sweeps(c, c.nu1, l));
  CyclePhase rs{};
  rs.op = PHASE_RESID;
  rs.n = D.ne;
  rs.cpl = D.cpl[prec];
  rs.mat = D.dia[prec];
  rs.perm = D.perm;
  rs.nbr = D.nbr;
  rs.tsc = scaled ? D.csc : nullptr;
  rs.rsc = scaled ? D.dsc : nullptr;
  rs.b = D.vb[vi];
  rs.x = D.vx[vi];
  rs.r = D.vr[vi];
  prog.push_back(rs);
  CyclePhase rt{};
  rt.op = PHASE_RESTRICT;
  rt.n = Dc.ne;
  rt.dims[0] = Dc.n[0];
  rt.dims[1] = Dc.n[1];
  rt.dims[2] = D.n[0];
  rt.dims[3] = D.n[1];
  rt.tr = c.child_P[vi];
  rt.in = D.vr[vi];
  rt.out = Dc.vb[vi];
  rt.xz = Dc.vx[vi];
  prog.push_back(rt);
  for (int v = coarse_visits(c, l); v > 0; --v) emit_cycle_phases(c, prec, l + 1, prog);
  CyclePhase pr{};
  pr.op = PHASE_PROLONG;
  pr.n = Dc.ne;
  pr.dims[0] = D.n[0];
  pr.dims[1] = D.n[1];
  pr.dims[2] = Dc.n[0];
  pr.dims[3] = Dc.n[1];
  pr.tr = c.child_PT[vi];
  pr.in = Dc.vx[vi];
  pr.out = D.vx[vi];
  prog.push_back(pr);
  smooth(level_sweeps(c, c.nu2, l));
}

void free_persist(Ctx& c) {
  for (int pr = 0; pr < 4; ++pr) {
    if (c.persist_prog[pr]) cudaFree(c.persist_prog[pr]);
    c.persist_prog[pr] = nullptr;
    c.persist_nphase[pr] = 0;
    c.persist_level[pr] = -1;
  }
}

// (Re)build the programs of the storage precisions the context runs cycles in
// (its cycle precision, and FP64), from the first level of at most
// persist_max elements below level 0; none when persist_max is 0.
void build_persist(Ctx& c) {
  free_persist(c);
  if (!c.ready || c.persist_max <= 0 || c.cut) return;
  const int L = nlevels(c);
  int l0 = -1;
  for (int l = 1; l < L; ++l)
    if (level_ne(c, l) <= c.persist_max) {
      l0 = l;
      break;
    }
  if (l0 < 0 || l0 >= L - 1) return;   // nothing to smooth below level 0 within the bound
  for (int pr : {c.precision, (int)STK_FP64}) {
    if (c.persist_prog[pr] || !c.dev[l0].cpl[pr] || !c.dev[l0].vx[pr == STK_FP64 ? 0 : 1]) continue;
    std::vector<CyclePhase> prog;
    emit_cycle_phases(c, pr, l0, prog);
    CyclePhase* d = nullptr;
    ck(cudaMalloc(&d, prog.size() * sizeof(CyclePhase)), "cudaMalloc program");
    ck(cudaMemcpy(d, prog.data(), prog.size() * sizeof(CyclePhase), cudaMemcpyHostToDevice), "copy program");
    c.persist_prog[pr] = d;
    c.persist_nphase[pr] = (int)prog.size();
    c.persist_level[pr] = l0;
  }
}

// Algorithm 1 on level 0 with 2 x 2 element clusters as the smoother's blocks
// (Concluding Remarks): b and x move to the cluster layout, the cluster
// records smooth and form the residual, which returns to the element layout
// for the restriction; the prolongation adds into the element layout of x.
void enqueue_cycle_clustered(Ctx& c, int prec, void* x, const void* b, cudaStream_t st) {
  const int vi = prec == STK_FP64 ? 0 : 1;
  DevLevel& D = c.dev[0];
  DevLevel& Dc = c.dev[1];
  DevLevel& K = c.cdev;
  const int n0 = D.n[0], n1 = D.n[1], nvar = c.d + 1;
  auto perm = [&](int to_cluster, const void* in, void* out) {
    ck(launch_cluster_permute(vi == 0, n0, n1, c.s, nvar, to_cluster, in, out, st), "cluster layout");
    c.launches++;
  };
  auto smooth = [&](int sweeps) {
    for (int it = 0; it < sweeps; ++it)
      for (int col = 0; col < K.ncolour; ++col) {
        const int n = K.cstart[col + 1] - K.cstart[col];
        if (n <= 0) continue;
        ck(run_element_on(c, c.cpat, K, prec, MODE_GS, K.cstart[col], n, K.inv[prec], c.cvb[vi], c.cvx[vi], nullptr,
                          st),
           "cluster colour step");
        c.launches++;
      }
  };
  perm(1, b, c.cvb[vi]);
  perm(1, x, c.cvx[vi]);
  smooth(level_sweeps(c, c.nu1, 0));
  ck(run_element_on(c, c.cpat, K, prec, MODE_RESID, 0, K.ne, K.dia[prec], c.cvb[vi], c.cvx[vi], c.cvr[vi], st),
     "cluster residual");
  c.launches++;
  perm(0, c.cvr[vi], D.vr[vi]);
  ck(launch_restrict(vi == 0, c.d, c.s, c.nb, Dc.n, D.n, Dc.ne, c.child_P[vi], D.vr[vi], Dc.vb[vi], st), "restrict");
  ck(cudaMemsetAsync(Dc.vx[vi], 0, (size_t)Dc.ne * c.nb * (vi == 0 ? 8 : 4), st), "memset");
  c.launches++;
  for (int v = coarse_visits(c, 0); v > 0; --v) enqueue_cycle(c, prec, 1, Dc.vx[vi], Dc.vb[vi], st);
  perm(0, c.cvx[vi], c.ctmp[vi]);
  ck(launch_prolong(vi == 0, c.d, c.s, c.nb, D.n, Dc.n, Dc.ne, c.child_PT[vi], Dc.vx[vi], c.ctmp[vi], st), "prolong");
  c.launches++;
  perm(1, c.ctmp[vi], c.cvx[vi]);
  smooth(level_sweeps(c, c.nu2, 0));
  perm(0, c.cvx[vi], x);
}

void enqueue_residual64(Ctx& c, const double* x, const double* b, double* r, cudaStream_t st) {
  DevLevel& D = c.dev[0];
  ck(run_element(c, 0, STK_FP64, MODE_RESID, 0, D.ne, D.dia[0], b, (void*)x, r, st), "residual64 launch");
  c.launches++;
}

void enqueue_norm(Ctx& c, const double* v, cudaStream_t st) {
  ck(launch_sumsq(level_ne(c, 0) * c.nb, v, c.norm_buf + 16, c.norm_buf, st), "norm launch");
  c.launches += 2;
  ck(cudaMemcpyAsync(c.norm_host, c.norm_buf, sizeof(double), cudaMemcpyDeviceToHost, st), "norm copy");
  ck(cudaMemcpyAsync(c.norm_host + 1, c.dev_err, sizeof(int), cudaMemcpyDeviceToHost, st), "flag copy");
}

// One outer iteration after the residual r64 of the current x is known:
// c = V(0, r), x += c, r64 = b - A x, ||r64||^2 -> host.
void enqueue_iteration(Ctx& c, double* x, const double* b, cudaStream_t st) {
  int prec = c.precision;
  int64_t n0 = level_ne(c, 0) * c.nb;
  DevLevel& D0 = c.dev[0];
  if (prec == STK_FP64) {
    ck(cudaMemsetAsync(c.c64, 0, n0 * 8, st), "memset");
    enqueue_cycle(c, prec, 0, c.c64, c.r64, st);
    ck(launch_axpy(1, 1, n0, x, c.c64, st), "axpy");
  } else {
    ck(launch_convert(0, 1, n0, D0.vb[1], c.r64, st), "convert");
    ck(cudaMemsetAsync(D0.vx[1], 0, n0 * 4, st), "memset");
    enqueue_cycle(c, prec, 0, D0.vx[1], D0.vb[1], st);
    ck(launch_axpy(1, 0, n0, x, D0.vx[1], st), "axpy");
    c.launches++;
  }
  c.launches++;
  enqueue_residual64(c, x, b, c.r64, st);
  enqueue_norm(c, c.r64, st);
}

// One outer iteration with the learned correction (low-precision cycle):
// c = V(0, r), delta from the cycle's residual, x += c + delta, r64 = b - A x,
// ||r64||^2 -> host.  The host then keeps or undoes delta (enqueue_undo).
void enqueue_learned_iteration(Ctx& c, double* x, const double* b, cudaStream_t st) {
  const int prec = c.precision;
  const int64_t n0 = level_ne(c, 0) * c.nb;
  DevLevel& D0 = c.dev[0];
  ck(launch_convert(0, 1, n0, D0.vb[1], c.r64, st), "convert");
  ck(cudaMemsetAsync(D0.vx[1], 0, n0 * 4, st), "memset");
  enqueue_cycle(c, prec, 0, D0.vx[1], D0.vb[1], st);
  enqueue_learned_delta(c, prec, D0.vx[1], D0.vb[1], st);
  ck(launch_axpy(1, 0, n0, x, D0.vx[1], st), "axpy");
  ck(launch_axpy(1, 0, n0, x, c.lxt, st), "axpy delta");
  c.launches += 3;
  enqueue_residual64(c, x, b, c.r64, st);
  enqueue_norm(c, c.r64, st);
}

// Undo the correction of the last learned iteration: x -= delta (leaving the
// plain cycle's result x + c), r64 = b - A x, ||r64||^2 -> host.
void enqueue_undo(Ctx& c, double* x, const double* b, cudaStream_t st) {
  const int64_t n0 = level_ne(c, 0) * c.nb;
  ck(launch_scale_f(n0, -1.f, c.lxt, c.lrt, st), "negate delta");
  ck(launch_axpy(1, 0, n0, x, c.lrt, st), "axpy -delta");
  c.launches += 2;
  enqueue_residual64(c, x, b, c.r64, st);
  enqueue_norm(c, c.r64, st);
}

// Capture what `enqueue` puts on st as an instantiated CUDA graph; the
// kernels it enqueued are counted into *kernels instead of c.launches.
template <typename F>
cudaGraphExec_t capture_graph(Ctx& c, cudaStream_t st, F&& enqueue, int64_t* kernels) {
  cudaGraph_t g;
  cudaGraphExec_t exec = nullptr;
  const int64_t before = c.launches;
  ck(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
  try {
    enqueue();
  } catch (...) {
    cudaStreamEndCapture(st, &g);
    c.launches = before;
    throw;
  }
  ck(cudaStreamEndCapture(st, &g), "end capture");
  cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  *kernels = c.launches - before;
  c.launches = before;
  ck(e, "graph instantiate");
  return exec;
}

bool valid_bc(const int* bc, int d) {
  for (int k = 0; k < d; ++k) {
    for (int sd = 0; sd < 2; ++sd)
      if (bc[2 * k + sd] < 0 || bc[2 * k + sd] > 2) return false;
    if ((bc[2 * k] == STK_BC_PERIODIC) != (bc[2 * k + 1] == STK_BC_PERIODIC)) return false;
  }
  return true;
}

int64_t count_points(const Ctx& c, int kind) {
  std::vector<double> xyz;
  face_points(c, kind, xyz, nullptr);
  return (int64_t)(xyz.size() / c.d);
}

// ---- several right-hand sides ----------------------------------------------------
void ensure_mrhs(Ctx& c, int nr) {
  if (c.mr_nr == nr) return;
  if (c.mgraph) cudaGraphExecDestroy(c.mgraph);
  c.mgraph = nullptr;
  c.mgraph_key[0] = -1;
  int L = nlevels(c);
  for (int l = 0; l < L; ++l) {
    DevLevel& D = c.dev[l];
    int64_t n = level_ne(c, l) * c.nb * nr;
    for (int v = 0; v < 2; ++v) {
      if (v == 1 && c.precision == STK_FP64) continue;
      size_t es = v == 0 ? 8 : 4;
      D.mx[v] = dalloc(c, n * es);
      D.mb[v] = dalloc(c, n * es);
      D.mr[v] = dalloc(c, n * es);
    }
  }
  int64_t m0 = level_ne(c, 0) * c.nb * nr;
  size_t ec = c.precision == STK_FP64 ? 8 : 4;
  c.mX = (double*)dalloc(c, m0 * 8);
  c.mB = (double*)dalloc(c, m0 * 8);
  c.mR = (double*)dalloc(c, m0 * 8);
  c.mRin = dalloc(c, m0 * ec);
  c.mRb = dalloc(c, m0 * ec);
  c.mAcc = dalloc(c, m0 * ec);
  c.mNorm = (double*)dalloc(c, 16 * 8);
  c.mPart = (double*)dalloc(c, 1024 * 8 * 8);
  c.mr_nr = nr;
}

void enqueue_cycle_mr(Ctx& c, int prec, int l, int nr, void* x, const void* b, cudaStream_t st) {
  int vi = prec == STK_FP64 ? 0 : 1;
  int L = nlevels(c);
  if (l == L - 1) {
    ck(launch_bottom_mr(vi == 0, c.nbot, nr, c.bottom_pinv, b, x, st), "bottom launch");
    c.launches++;
    return;
  }
  DevLevel& D = c.dev[l];
  DevLevel& Dc = c.dev[l + 1];
  auto smooth = [&](int sweeps) {
    for (int it = 0; it < sweeps; ++it)
      for (int col = 0; col < D.ncolour; ++col) {
        int n = D.cstart[col + 1] - D.cstart[col];
        if (n <= 0) continue;
        ck(launch_element_mrhs(c.pat, prec, nr, MODE_GS, D.cstart[col], n, D.perm, D.nbr, D.cpl[prec], D.inv[prec],
                               b, x, nullptr, st, c.mrhs_tensor, c.wide_max),
           "gs launch");
        c.launches++;
      }
  };
  smooth(level_sweeps(c, c.nu1, l));
  ck(launch_element_mrhs(c.pat, prec, nr, MODE_RESID, 0, D.ne, D.perm, D.nbr, D.cpl[prec], D.dia[prec], b, x,
                         D.mr[vi], st, c.mrhs_tensor, c.wide_max),
     "residual launch");
  ck(launch_restrict_mr(vi == 0, c.d, c.s, c.nb, nr, Dc.n, D.n, Dc.ne, c.child_P[vi], D.mr[vi], Dc.mb[vi], st),
     "restrict launch");
  ck(cudaMemsetAsync(Dc.mx[vi], 0, (size_t)Dc.ne * c.nb * nr * (vi == 0 ? 8 : 4), st), "memset");
  c.launches += 2;
  for (int v = coarse_visits(c, l); v > 0; --v) enqueue_cycle_mr(c, prec, l + 1, nr, Dc.mx[vi], Dc.mb[vi], st);
  ck(launch_prolong_mr(vi == 0, c.d, c.s, c.nb, nr, D.n, Dc.n, Dc.ne, c.child_PT[vi], Dc.mx[vi], x, st),
     "prolong launch");
  c.launches++;
  smooth(level_sweeps(c, c.nu2, l));
}

// One outer iteration on the interleaved level-0 FP64 vectors mX, mB:
// mR = mB - A mX (FP64); Rb = mR in cycle precision; Acc = 0; then `inner`
// times: Rin = Rb - A Acc (cycle precision; Rin = Rb the first time),
// Acc += V(0, Rin); finally mX += Acc and the squared norms of the new
// residual are left in mNorm / norm_host.
void enqueue_mr_iteration(Ctx& c, int nr, int inner, cudaStream_t st) {
  int prec = c.precision, vi = prec == STK_FP64 ? 0 : 1;
  int64_t m0 = level_ne(c, 0) * c.nb * nr;
  DevLevel& D0 = c.dev[0];
  size_t ec = vi == 0 ? 8 : 4;
  ck(launch_convert(vi == 0, 1, m0, c.mRb, c.mR, st), "convert");
  ck(cudaMemsetAsync(c.mAcc, 0, m0 * ec, st), "memset");
  c.launches++;
  for (int k = 0; k < inner; ++k) {
    const void* rin = c.mRb;
    if (k > 0) {
      ck(launch_element_mrhs(c.pat, prec, nr, MODE_RESID, 0, D0.ne, D0.perm, D0.nbr, D0.cpl[prec], D0.dia[prec],
                             c.mRb, c.mAcc, c.mRin, st, c.mrhs_tensor, c.wide_max),
         "inner residual");
      c.launches++;
      rin = c.mRin;
    }
    ck(cudaMemsetAsync(D0.mx[vi], 0, m0 * ec, st), "memset");
    enqueue_cycle_mr(c, prec, 0, nr, D0.mx[vi], rin, st);
    ck(launch_axpy(vi == 0, vi == 0, m0, c.mAcc, D0.mx[vi], st), "axpy");
    c.launches++;
  }
  ck(launch_axpy(1, vi == 0, m0, c.mX, c.mAcc, st), "axpy");
  c.launches++;
  ck(launch_element_mrhs(c.pat, STK_FP64, nr, MODE_RESID, 0, D0.ne, D0.perm, D0.nbr, D0.cpl[0], D0.dia[0], c.mB, c.mX,
                         c.mR, st, c.mrhs_tensor, c.wide_max),
     "residual64");
  ck(launch_sumsq_mr(level_ne(c, 0) * c.nb, nr, c.mR, c.mPart, c.mNorm, st), "norms");
  c.launches += 3;
  ck(cudaMemcpyAsync(c.norm_host, c.mNorm, nr * sizeof(double), cudaMemcpyDeviceToHost, st), "norm copy");
}

// ---- lockstep flexible GMRES for several right-hand sides ----------------------
// nr Krylov sequences advance together on interleaved vectors: one multi-RHS
// V-cycle per Arnoldi step preconditions all of them (one record stream for
// nr products), one FP64 multi-RHS residual kernel forms A z for all of
// them; dots, norms and Givens rotations stay per right-hand side.  A
// right-hand side that has converged keeps zero basis vectors from then on.
void ensure_krylov_mr(Ctx& c, int nr, int m) {
  if (c.mkV && c.mk_cap >= m && c.mk_nr == nr) return;
  const int64_t n = level_ne(c, 0) * c.nb * nr;
  c.mkV = (double*)dalloc(c, (size_t)(m + 1) * n * 8);
  c.mkZ = (double*)dalloc(c, (size_t)m * n * 8);
  c.mkw = (double*)dalloc(c, (size_t)n * 8);
  c.mkzero = (double*)dalloc(c, (size_t)n * 8);
  ck(cudaMemset(c.mkzero, 0, (size_t)n * 8), "memset");
  c.mkpart = (double*)dalloc(c, (size_t)1024 * 256 * 8);
  c.mkdev = (double*)dalloc(c, 3 * 256 * 8);
  if (!c.mkhost) ck(cudaMallocHost(&c.mkhost, 3 * 256 * sizeof(double)), "cudaMallocHost");
  if (c.precision != STK_FP64) {
    c.mkz32 = (float*)dalloc(c, (size_t)n * 4);
    c.mkw32 = (float*)dalloc(c, (size_t)n * 4);
    c.mkzero32 = (float*)dalloc(c, (size_t)n * 4);
    ck(cudaMemset(c.mkzero32, 0, (size_t)n * 4), "memset");
  }
  c.mk_cap = m;
  c.mk_nr = nr;
}

// z = V(0, v) for all right-hand sides (FP64 interleaved in and out).
void precondition_mr(Ctx& c, int nr, const double* v, double* z, cudaStream_t st) {
  const int prec = c.precision, vi = prec == STK_FP64 ? 0 : 1;
  const int64_t n = level_ne(c, 0) * c.nb * nr;
  DevLevel& D0 = c.dev[0];
  if (vi == 0) {
    ck(cudaMemsetAsync(z, 0, (size_t)n * 8, st), "memset");
    enqueue_cycle_mr(c, prec, 0, nr, z, v, st);
    return;
  }
  ck(launch_convert(0, 1, n, c.mRin, v, st), "convert");
  ck(cudaMemsetAsync(D0.mx[1], 0, (size_t)n * 4, st), "memset");
  enqueue_cycle_mr(c, prec, 0, nr, D0.mx[1], c.mRin, st);
  ck(launch_convert(1, 0, n, z, D0.mx[1], st), "convert");
  c.launches += 2;
}

// out[i * nr + q] = V_i . w over right-hand side q, i < k (host copy).
void mr_dots(Ctx& c, int nr, int k, const double* V, const double* w, double* out, cudaStream_t st) {
  const int64_t n = level_ne(c, 0) * c.nb * nr;
  ck(launch_multidot_mr(n, nr, k, V, n, w, c.mkpart, c.mkdev, st), "multidot");
  c.launches += 2;
  ck(cudaMemcpyAsync(c.mkhost, c.mkdev, (size_t)k * nr * 8, cudaMemcpyDeviceToHost, st), "copy dots");
  ck(cudaStreamSynchronize(st), "sync");
  std::copy(c.mkhost, c.mkhost + (size_t)k * nr, out);
}

// w = alpha w + sum_i coef[i * nr + q] V_i (per right-hand side q).
void mr_axpy(Ctx& c, int nr, int k, double alpha, const double* coef, const double* V, double* w, cudaStream_t st) {
  const int64_t n = level_ne(c, 0) * c.nb * nr;
  double* hc = c.mkhost + 256;
  std::copy(coef, coef + (size_t)k * nr, hc);
  ck(cudaMemcpyAsync(c.mkdev + 256, hc, (size_t)std::max(k * nr, 1) * 8, cudaMemcpyHostToDevice, st), "copy coef");
  ck(launch_multiaxpy_mr(n, nr, k, alpha, c.mkdev + 256, V, n, w, st), "multiaxpy");
  c.launches++;
  ck(cudaStreamSynchronize(st), "sync");   // hc is reused by the next call
}

// y = s[q] x (per right-hand side q).
void mr_scale(Ctx& c, int nr, const double* sc, const double* x, double* y, cudaStream_t st) {
  const int64_t n = level_ne(c, 0) * c.nb * nr;
  double* hs = c.mkhost + 512;
  std::copy(sc, sc + nr, hs);
  ck(cudaMemcpyAsync(c.mkdev + 512, hs, (size_t)nr * 8, cudaMemcpyHostToDevice, st), "copy scales");
  ck(launch_scale_mr(n, nr, c.mkdev + 512, x, y, st), "scale");
  c.launches++;
  ck(cudaStreamSynchronize(st), "sync");
}

// squared norms per right-hand side (host copy, nr entries).
void mr_norms(Ctx& c, int nr, const double* v, double* out, cudaStream_t st) {
  ck(launch_sumsq_mr(level_ne(c, 0) * c.nb, nr, v, c.mPart, c.mNorm, st), "norms");
  c.launches += 2;
  ck(cudaMemcpyAsync(c.mkhost + 768 - 16, c.mNorm, (size_t)nr * 8, cudaMemcpyDeviceToHost, st), "copy norms");
  ck(cudaStreamSynchronize(st), "sync");
  std::copy(c.mkhost + 768 - 16, c.mkhost + 768 - 16 + nr, out);
}

// On entry c.mR = B - A X and rel[q] its relative norms; returns the number
// of Arnoldi steps, X (c.mX) updated and rel[q] the final true residuals.
int fgmres_mr(Ctx& c, int nr, int nrhs, double rtol, int maxit, double* hist, const std::vector<double>& bn,
              std::vector<double>& rel, cudaStream_t st) {
  const int m = std::max(1, std::min(c.restart, 256 / nr));
  ensure_krylov_mr(c, nr, m);
  // refined variant: FP32 Krylov matvec, each right-hand side's cycle trusted
  // for a 1e-5 reduction before the FP64 residual restarts it
  const bool refined = c.solver == 2 && c.precision != STK_FP64;
  const int64_t n = level_ne(c, 0) * c.nb * nr;
  DevLevel& D0 = c.dev[0];
  std::vector<double> H((size_t)nr * (m + 1) * m), g((size_t)nr * (m + 1)), cs((size_t)nr * m),
      sn((size_t)nr * m), h((size_t)(m + 1) * nr), h2((size_t)(m + 1) * nr), coef((size_t)(m + 1) * nr),
      hn(nr), scl(nr), beta(nr);
  std::vector<int> kq(nr, 0);
  std::vector<char> active(nr, 0);
  auto Hq = [&](int q, int i, int j) -> double& { return H[((size_t)q * (m + 1) + i) * m + j]; };
  int it = 0;
  auto any_left = [&]() {
    for (int q = 0; q < nrhs; ++q)
      if (!(rel[q] <= rtol)) return true;
    return false;
  };
  while (any_left() && it < maxit) {
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    for (int q = 0; q < nr; ++q) {
      beta[q] = rel[q] * (q < nrhs ? bn[q] : 0.0);
      active[q] = q < nrhs && !(rel[q] <= rtol) && beta[q] > 0;
      scl[q] = active[q] ? 1.0 / beta[q] : 0.0;
      g[(size_t)q * (m + 1)] = active[q] ? beta[q] : 0.0;
      kq[q] = 0;
    }
    mr_scale(c, nr, scl.data(), c.mR, c.mkV, st);
    int k = 0;
    for (int j = 0; j < m && it < maxit; ++j) {
      double* vj = c.mkV + (size_t)j * n;
      double* zj = c.mkZ + (size_t)j * n;
      precondition_mr(c, nr, vj, zj, st);
      // w' = 0 - A z_j (FP64, or FP32 blocks and vectors in the refined
      // variant); classical Gram-Schmidt twice on w = -w'
      if (refined) {
        ck(launch_convert(0, 1, n, c.mkz32, zj, st), "convert");
        ck(launch_element_mrhs(c.pat, STK_FP32, nr, MODE_RESID, 0, D0.ne, D0.perm, D0.nbr, D0.cpl[STK_FP32],
                               D0.dia[STK_FP32], c.mkzero32, c.mkz32, c.mkw32, st, 0),   // exact FP32 sums
           "matvec32");
        ck(launch_convert(1, 0, n, c.mkw, c.mkw32, st), "convert");
        c.launches += 3;
      } else {
        ck(launch_element_mrhs(c.pat, STK_FP64, nr, MODE_RESID, 0, D0.ne, D0.perm, D0.nbr, D0.cpl[0], D0.dia[0],
                               c.mkzero, zj, c.mkw, st, c.mrhs_tensor, c.wide_max),
           "matvec64");
        c.launches++;
      }
      mr_dots(c, nr, j + 1, c.mkV, c.mkw, h.data(), st);
      for (size_t u = 0; u < (size_t)(j + 1) * nr; ++u) {
        h[u] = -h[u];
        coef[u] = -h[u];
      }
      mr_axpy(c, nr, j + 1, -1.0, coef.data(), c.mkV, c.mkw, st);
      mr_dots(c, nr, j + 1, c.mkV, c.mkw, h2.data(), st);
      for (size_t u = 0; u < (size_t)(j + 1) * nr; ++u) {
        h[u] += h2[u];
        coef[u] = -h2[u];
      }
      mr_axpy(c, nr, j + 1, 1.0, coef.data(), c.mkV, c.mkw, st);
      mr_norms(c, nr, c.mkw, hn.data(), st);
      for (int q = 0; q < nr; ++q) {
        hn[q] = std::sqrt(hn[q]);
        scl[q] = active[q] && hn[q] > 0 && std::isfinite(hn[q]) ? 1.0 / hn[q] : 0.0;
      }
      mr_scale(c, nr, scl.data(), c.mkw, c.mkV + (size_t)(j + 1) * n, st);
      ++it;
      k = j + 1;
      for (int q = 0; q < nrhs; ++q) {
        if (!active[q]) {
          if (hist) hist[(size_t)it * nrhs + q] = rel[q];
          continue;
        }
        if (!std::isfinite(hn[q])) {
          rel[q] = hn[q];
          return it;
        }
        for (int i = 0; i <= j; ++i) Hq(q, i, j) = h[(size_t)i * nr + q];
        Hq(q, j + 1, j) = hn[q];
        double* gq = &g[(size_t)q * (m + 1)];
        double* cq = &cs[(size_t)q * m];
        double* sq = &sn[(size_t)q * m];
        for (int i = 0; i < j; ++i) {
          const double a = Hq(q, i, j), bb = Hq(q, i + 1, j);
          Hq(q, i, j) = cq[i] * a + sq[i] * bb;
          Hq(q, i + 1, j) = -sq[i] * a + cq[i] * bb;
        }
        const double a = Hq(q, j, j), bb = Hq(q, j + 1, j);
        const double den = std::hypot(a, bb);
        cq[j] = den > 0 ? a / den : 1.0;
        sq[j] = den > 0 ? bb / den : 0.0;
        Hq(q, j, j) = den;
        Hq(q, j + 1, j) = 0.0;
        gq[j + 1] = -sq[j] * gq[j];
        gq[j] = cq[j] * gq[j];
        kq[q] = j + 1;
        rel[q] = std::fabs(gq[j + 1]) / bn[q];
        if (hist) hist[(size_t)it * nrhs + q] = rel[q];
        if (rel[q] <= rtol || (refined && std::fabs(gq[j + 1]) <= 1e-5 * beta[q])) active[q] = 0;
      }
      bool any = false;
      for (int q = 0; q < nrhs; ++q) any = any || active[q];
      if (!any) break;
    }
    // X += Z y_q per right-hand side, y_q from its own triangular system
    std::fill(coef.begin(), coef.end(), 0.0);
    for (int q = 0; q < nrhs; ++q) {
      const int kk = kq[q];
      const double* gq = &g[(size_t)q * (m + 1)];
      std::vector<double> y(kk);
      for (int i = kk - 1; i >= 0; --i) {
        double acc = gq[i];
        for (int jj = i + 1; jj < kk; ++jj) acc -= Hq(q, i, jj) * y[jj];
        y[i] = Hq(q, i, i) != 0 ? acc / Hq(q, i, i) : 0.0;
      }
      for (int i = 0; i < kk; ++i) coef[(size_t)i * nr + q] = y[i];
    }
    mr_axpy(c, nr, k, 1.0, coef.data(), c.mkZ, c.mX, st);
    // true FP64 residual and its norms
    ck(launch_element_mrhs(c.pat, STK_FP64, nr, MODE_RESID, 0, D0.ne, D0.perm, D0.nbr, D0.cpl[0], D0.dia[0], c.mB,
                           c.mX, c.mR, st, c.mrhs_tensor, c.wide_max),
       "residual64");
    c.launches++;
    std::vector<double> r2(nr);
    mr_norms(c, nr, c.mR, r2.data(), st);
    for (int q = 0; q < nrhs; ++q) {
      rel[q] = std::sqrt(r2[q]) / bn[q];
      if (hist) hist[(size_t)it * nrhs + q] = rel[q];
      if (!std::isfinite(rel[q])) return it;
    }
  }
  return it;
}

// ---- flexible GMRES with the V-cycle as right preconditioner ----------------
// Krylov buffers for m basis directions (m+1 vectors of V, m of Z).
void ensure_krylov(Ctx& c, int m) {
  if (c.kcap >= m && c.kV) return;
  int64_t n0 = level_ne(c, 0) * c.nb;
  c.kV = (double*)dalloc(c, (size_t)(m + 1) * n0 * 8);
  c.kZ = (double*)dalloc(c, (size_t)m * n0 * 8);
  c.kw = (double*)dalloc(c, (size_t)n0 * 8);
  c.kzero = (double*)dalloc(c, (size_t)n0 * 8);
  ck(cudaMemset(c.kzero, 0, (size_t)n0 * 8), "memset");
  c.kpart = (double*)dalloc(c, (size_t)1024 * 136 * 8);
  if (c.precision != STK_FP64) {
    c.kz32 = (float*)dalloc(c, (size_t)n0 * 4);
    c.kw32 = (float*)dalloc(c, (size_t)n0 * 4);
    c.kzero32 = (float*)dalloc(c, (size_t)n0 * 4);
    ck(cudaMemset(c.kzero32, 0, (size_t)n0 * 4), "memset");
  }
  c.kdots = (double*)dalloc(c, 272 * 8);
  if (!c.khost) ck(cudaMallocHost(&c.khost, 272 * sizeof(double)), "cudaMallocHost");
  c.kcap = m;
}

// The V-cycle on the level-0 work vectors (b0 -> x0, x0 zeroed first) as a graph.
void ensure_cycle_graph(Ctx& c, cudaStream_t st) {
  if (c.cycle_graph && c.cycle_graph_prec == c.precision) return;
  if (c.cycle_graph) cudaGraphExecDestroy(c.cycle_graph);
  c.cycle_graph = nullptr;
  int vi = c.precision == STK_FP64 ? 0 : 1;
  DevLevel& D0 = c.dev[0];
  int64_t n0 = level_ne(c, 0) * c.nb;
  cudaGraph_t g;
  int64_t before = c.launches;
  ck(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
  try {
    ck(cudaMemsetAsync(D0.vx[vi], 0, (size_t)n0 * (vi == 0 ? 8 : 4), st), "memset");
    enqueue_cycle(c, c.precision, 0, D0.vx[vi], D0.vb[vi], st);
  } catch (...) {
    cudaStreamEndCapture(st, &g);
    c.launches = before;
    throw;
  }
  ck(cudaStreamEndCapture(st, &g), "end capture");
  ck(cudaGraphInstantiate(&c.cycle_graph, g, 0), "graph instantiate");
  cudaGraphDestroy(g);
  c.cycle_graph_kernels = c.launches - before;
  c.launches = before;
  c.cycle_graph_prec = c.precision;
}

// z = V(0, v): one V-cycle of the configured precision from a zero guess.
void precondition(Ctx& c, const double* v, double* z, cudaStream_t st) {
  int64_t n0 = level_ne(c, 0) * c.nb;
  DevLevel& D0 = c.dev[0];
  if (c.precision == STK_FP64) {
    ck(cudaMemcpyAsync(D0.vb[0], v, (size_t)n0 * 8, cudaMemcpyDeviceToDevice, st), "copy");
  } else {
    ck(launch_convert(0, 1, n0, D0.vb[1], v, st), "convert");
    c.launches++;
  }
  ck(cudaGraphLaunch(c.cycle_graph, st), "cycle graph");
  c.launches += c.cycle_graph_kernels;
  if (c.precision == STK_FP64) {
    ck(cudaMemcpyAsync(z, D0.vx[0], (size_t)n0 * 8, cudaMemcpyDeviceToDevice, st), "copy");
  } else {
    ck(launch_convert(1, 0, n0, z, D0.vx[1], st), "convert");
    c.launches++;
  }
}

// h[0..k) = V[0..k)^T w on the host.
void host_dots(Ctx& c, int k, const double* V, const double* w, double* h, cudaStream_t st) {
  int64_t n0 = level_ne(c, 0) * c.nb;
  ck(launch_multidot(n0, k, V, n0, w, c.kpart, c.kdots, st), "multidot");
  c.launches += 2;
  ck(cudaMemcpyAsync(c.khost, c.kdots, (size_t)k * 8, cudaMemcpyDeviceToHost, st), "copy dots");
  ck(cudaStreamSynchronize(st), "sync");
  std::copy(c.khost, c.khost + k, h);
}

// w = alpha w + sum_i coef[i] V[i] (coef from the host).
void host_axpy(Ctx& c, int k, double alpha, const double* coef, const double* V, double* w, cudaStream_t st) {
  int64_t n0 = level_ne(c, 0) * c.nb;
  double* hc = c.khost + 136;
  std::copy(coef, coef + k, hc);
  ck(cudaMemcpyAsync(c.kdots + 136, hc, (size_t)std::max(k, 1) * 8, cudaMemcpyHostToDevice, st), "copy coef");
  ck(launch_multiaxpy(n0, k, alpha, c.kdots + 136, V, n0, w, st), "multiaxpy");
  c.launches++;
  ck(cudaStreamSynchronize(st), "sync");   // hc is reused by the next call
}

struct Timeout {};

double host_norm(Ctx& c, const double* v, cudaStream_t st) {
  enqueue_norm(c, v, st);
  ck(cudaStreamSynchronize(st), "sync");
  if (reinterpret_cast<int*>(c.norm_host + 1)[0] != 0) throw Timeout{};
  return std::sqrt(c.norm_host[0]);
}

// Returns the iteration count; rel holds the final true relative residual.
// On entry c.r64 holds b - A x and rel its norm over bnorm (stk_solve).
int fgmres(Ctx& c, double* x, const double* b, double rtol, int maxit, double* hist, double bnorm,
           double& rel, cudaStream_t st) {
  ensure_krylov(c, c.restart);
  ensure_cycle_graph(c, st);
  int64_t n0 = level_ne(c, 0) * c.nb;
  const int m = c.restart;
  std::vector<double> H((size_t)(m + 1) * m), g(m + 1), cs(m), sn(m), h(m + 1), h2(m + 1), y(m);
  double beta = rel * bnorm;
  double rel0 = rel;
  int it = 0;
  while (rel > rtol && it < maxit) {
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    ck(launch_scale(n0, 1.0 / beta, c.r64, c.kV, st), "scale");
    c.launches++;
    int k = 0;
    for (int j = 0; j < m && it < maxit; ++j) {
      double* vj = c.kV + (size_t)j * n0;
      double* zj = c.kZ + (size_t)j * n0;
      precondition(c, vj, zj, st);
      // w = A z_j, computed as -(0 - A z_j) by the residual kernel; in the
      // refined variant with FP32 blocks (FP32 vectors, FP32 accumulation).
      if (c.solver == 2 && c.precision != STK_FP64) {
        ck(launch_convert(0, 1, n0, c.kz32, zj, st), "convert");
        ck(run_element(c, 0, STK_FP32, MODE_RESID, 0, c.dev[0].ne, c.dev[0].dia[STK_FP32], c.kzero32, c.kz32,
                       c.kw32, st),
           "matvec32");
        ck(launch_convert(1, 0, n0, c.kw, c.kw32, st), "convert");
        c.launches += 3;
      } else if (c.precision != STK_FP64 && c.df_matvec && c.dev[0].cpl_lo) {
        // z_j is an FP32 vector (the cycle's output, still in vx[1]): -A z_j to
        // about 2^-44 with FP32 records and remainders on the FP32 units
        DevLevel& D0 = c.dev[0];
        ck(launch_element_df(c.pat, 0, D0.ne, D0.perm, D0.nbr, D0.cpl[STK_FP32], D0.cpl_lo, D0.dia[STK_FP32],
                             D0.dia_lo, (const float*)D0.vx[1], c.kw, c.warp_ctas[STK_FP32], st),
           "matvec df");
        c.launches++;
      } else {
        enqueue_residual64(c, zj, c.kzero, c.kw, st);
      }
      // Classical Gram-Schmidt, twice.
      host_dots(c, j + 1, c.kV, c.kw, h.data(), st);
      for (int i = 0; i <= j; ++i) h[i] = -h[i];
      std::vector<double> negh(j + 1);
      for (int i = 0; i <= j; ++i) negh[i] = -h[i];
      host_axpy(c, j + 1, -1.0, negh.data(), c.kV, c.kw, st);
      host_dots(c, j + 1, c.kV, c.kw, h2.data(), st);
      for (int i = 0; i <= j; ++i) {
        negh[i] = -h2[i];
        h[i] += h2[i];
      }
      host_axpy(c, j + 1, 1.0, negh.data(), c.kV, c.kw, st);
      double hn = host_norm(c, c.kw, st);
      if (!std::isfinite(hn)) {
        rel = hn;
        return it + 1;
      }
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h[i];
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0) {
        ck(launch_scale(n0, 1.0 / hn, c.kw, c.kV + (size_t)(j + 1) * n0, st), "scale");
        c.launches++;
      }
      for (int i = 0; i < j; ++i) {
        double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
      double den = std::hypot(a, bb);
      cs[j] = a / den;
      sn[j] = bb / den;
      H[(size_t)j * m + j] = den;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      k = j + 1;
      ++it;
      rel = std::fabs(g[j + 1]) / bnorm;
      if (hist) hist[it] = rel;
      if (rel <= rtol || !std::isfinite(rel) || rel > 1e6 * rel0) break;
      // Refined variant: the low-precision Krylov relation is trusted for a
      // 1e-5 reduction, then x is updated and the FP64 residual restarts it.
      if (c.solver == 2 && std::fabs(g[j + 1]) <= 1e-5 * beta) break;
    }
    // x += Z y with H[:k,:k] y = g[:k]
    for (int i = k - 1; i >= 0; --i) {
      double acc = g[i];
      for (int jj = i + 1; jj < k; ++jj) acc -= H[(size_t)i * m + jj] * y[jj];
      y[i] = acc / H[(size_t)i * m + i];
    }
    host_axpy(c, k, 1.0, y.data(), c.kZ, x, st);
    enqueue_residual64(c, x, b, c.r64, st);
    beta = host_norm(c, c.r64, st);
    rel = beta / bnorm;
    if (hist) hist[it] = rel;
    if (!std::isfinite(rel) || rel > 1e6 * rel0) break;
  }
  return it;
}

// eq. (rho): GMRES, not restarted, on the left-preconditioned system
// V A x = V b with b = 0 from x0 (Section 4), V = one cycle of the context's
// precision from a zero guess.  The preconditioned residual r_k = -V A x_k is
// minimised over x0 + K_k(V A, r0); stops at the first n with
// ||r_n|| <= reduction ||r_0|| or at maxit.  hist[k] = ||r_k|| / ||r_0||;
// hess (optional) gets the Arnoldi matrix H (row-major, (maxit+1) x maxit)
// before the Givens rotations, whose leading n x n block's eigenvalues
// estimate the spectrum of V A (Section 4's spectral estimate).
int gmres_rho(Ctx& c, const double* x0, double reduction, int maxit, double* hist, double* hess, double& rho,
              cudaStream_t st) {
  ensure_krylov(c, maxit);
  ensure_cycle_graph(c, st);
  const int64_t n0 = level_ne(c, 0) * c.nb;
  const int m = maxit;
  std::vector<double> H((size_t)(m + 1) * m, 0.0), g(m + 1, 0.0), cs(m), sn(m), h(m + 1), h2(m + 1), negh(m + 1);
  // r0 = V(0 - A x0) = -V A x0
  enqueue_residual64(c, x0, c.kzero, c.kw, st);
  precondition(c, c.kw, c.kV, st);
  const double beta = host_norm(c, c.kV, st);
  if (hist) hist[0] = 1.0;
  if (!(beta > 0) || !std::isfinite(beta)) {
    rho = std::isfinite(beta) ? 0.0 : beta;   // x0 in the kernel: rho 0; NaN / Inf reported
    return 0;
  }
  ck(launch_scale(n0, 1.0 / beta, c.kV, c.kV, st), "scale");
  c.launches++;
  g[0] = beta;
  int n = 0;
  for (int j = 0; j < m; ++j) {
    double* vj = c.kV + (size_t)j * n0;
    double* w = c.kV + (size_t)(j + 1) * n0;
    // w = V A v_j: the residual kernel forms -A v_j, the cycle is linear
    enqueue_residual64(c, vj, c.kzero, c.kw, st);
    precondition(c, c.kw, w, st);
    ck(launch_scale(n0, -1.0, w, w, st), "scale");
    c.launches++;
    // classical Gram-Schmidt, twice
    host_dots(c, j + 1, c.kV, w, h.data(), st);
    for (int i = 0; i <= j; ++i) negh[i] = -h[i];
    host_axpy(c, j + 1, 1.0, negh.data(), c.kV, w, st);
    host_dots(c, j + 1, c.kV, w, h2.data(), st);
    for (int i = 0; i <= j; ++i) {
      negh[i] = -h2[i];
      h[i] += h2[i];
    }
    host_axpy(c, j + 1, 1.0, negh.data(), c.kV, w, st);
    const double hn = host_norm(c, w, st);
    for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h[i];
    H[(size_t)(j + 1) * m + j] = hn;
    if (hess)
      for (int i = 0; i <= j + 1; ++i) hess[(size_t)i * m + j] = H[(size_t)i * m + j];
    if (hn > 0) {
      ck(launch_scale(n0, 1.0 / hn, w, w, st), "scale");
      c.launches++;
    }
    for (int i = 0; i < j; ++i) {
      const double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
      H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
      H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
    }
    const double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
    const double den = std::hypot(a, bb);
    cs[j] = a / den;
    sn[j] = bb / den;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    n = j + 1;
    if (hist) hist[n] = std::fabs(g[n]) / beta;
    if (!std::isfinite(g[n]) || std::fabs(g[n]) <= reduction * beta || hn == 0) break;
  }
  rho = std::exp(std::log(std::fabs(g[n]) / beta) / n);
  return n;
}

}  // namespace

extern "C" {

int stk_create(stk_ctx** out, int device) {
  if (!out) return STK_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return STK_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return STK_ERR_CUDA;
  stk_ctx* c = new (std::nothrow) stk_ctx();
  if (!c) return STK_ERR_OOM;
  c->device = device;
  if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return STK_ERR_CUDA;
  }
  *out = c;
  return STK_OK;
}

int stk_destroy(stk_ctx* c) {
  if (!c) return STK_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  free_device(*c);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return STK_OK;
}

const char* stk_last_error(stk_ctx* c) { return c ? c->err.c_str() : "null context"; }

int stk_set_mesh(stk_ctx* c, int d, const int* n, const double* lo, const double* hi, const int* bc) {
  return guard(c, [&]() -> int {
    if (d < 2 || d > 3 || !n || !lo || !hi || !bc) return fail(c, STK_ERR_INVALID_ARG, "bad mesh arguments");
    for (int k = 0; k < d; ++k) {
      if (n[k] < 1 || !(hi[k] > lo[k])) return fail(c, STK_ERR_INVALID_ARG, "bad mesh extent");
    }
    if (!valid_bc(bc, d)) return fail(c, STK_ERR_INVALID_ARG, "bad boundary types");
    free_device(*c);
    c->host.clear();
    c->d = d;
    for (int k = 0; k < 3; ++k) {
      c->n[k] = k < d ? n[k] : 1;
      c->lo[k] = k < d ? lo[k] : 0.0;
      c->hi[k] = k < d ? hi[k] : 1.0;
    }
    for (int i = 0; i < 6; ++i) c->bc[i] = i < 2 * d ? bc[i] : 0;
    c->mu_vol.clear();
    return STK_OK;
  });
}

int stk_set_discretisation(stk_ctx* c, int p, int gamma) {
  return guard(c, [&]() -> int {
    if (c->d == 0) return fail(c, STK_ERR_INVALID_ARG, "set the mesh first");
    if (p < 1 || (gamma != 0 && gamma != 1)) return fail(c, STK_ERR_INVALID_ARG, "bad degree or form");
    int s = 1;
    for (int k = 0; k < c->d; ++k) s *= (p + 1);
    if (!(s == 4 || s == 8 || s == 9 || s == 16 || s == 25 || s == 27))
      return fail(c, STK_ERR_INVALID_ARG, "unsupported (d, p): supported 2D p=1..4, 3D p=1..2");
    free_device(*c);
    c->p = p;
    c->gamma = gamma;
    c->s = s;
    c->nb = (c->d + 1) * s;
    c->q = 2 * p + 2;
    if (c->tau0 < 0) c->tau0 = 0.5 * p;
    build_pattern(c->d, p, gamma, false, c->pat);
    c->chi.clear();
    c->mu_phase.clear();
    c->mu_vol.clear();
    return STK_OK;
  });
}

int stk_set_penalty(stk_ctx* c, double tau, double tau0, double c_bdry, double c_intra) {
  return guard(c, [&]() -> int {
    if (!(tau > 0) || !(tau0 > 0) || !(c_bdry >= 0) || !(c_intra >= 0))
      return fail(c, STK_ERR_INVALID_ARG, "penalties must be positive");
    c->tau = tau;
    c->tau0 = tau0;
    c->c_bdry = c_bdry;
    c->c_intra = c_intra;
    return STK_OK;
  });
}

int stk_num_points(stk_ctx* c, int kind, int64_t* count) {
  return guard(c, [&]() -> int {
    if (c->p < 0 || !count || kind < 0 || kind > (c->cut ? 3 : 2)) return fail(c, STK_ERR_INVALID_ARG, "bad call");
    *count = c->cut ? cut_count_points(*c, kind) : count_points(*c, kind);
    return STK_OK;
  });
}

int stk_get_point_phases(stk_ctx* c, int kind, int* phase) {
  return guard(c, [&]() -> int {
    if (c->p < 0 || !phase || kind < 0 || kind > (c->cut ? 3 : 2)) return fail(c, STK_ERR_INVALID_ARG, "bad call");
    if (!c->cut) return fail(c, STK_ERR_INVALID_ARG, "point phases belong to cut-cell meshes");
    std::vector<double> pts;
    std::vector<int> ph;
    cut_points(*c, kind, pts, nullptr, &ph);
    std::copy(ph.begin(), ph.end(), phase);
    return STK_OK;
  });
}

int stk_get_points(stk_ctx* c, int kind, double* xyz, double* normals) {
  return guard(c, [&]() -> int {
    if (c->p < 0 || !xyz || kind < 0 || kind > (c->cut ? 3 : 2)) return fail(c, STK_ERR_INVALID_ARG, "bad call");
    if (c->cut) {
      std::vector<double> pts, nrm;
      cut_points(*c, kind, pts, normals ? &nrm : nullptr, nullptr);
      std::copy(pts.begin(), pts.end(), xyz);
      if (normals) std::copy(nrm.begin(), nrm.end(), normals);
      return STK_OK;
    }
    std::vector<double> pts, nrm;
    face_points(*c, kind, pts, normals ? &nrm : nullptr);
    std::copy(pts.begin(), pts.end(), xyz);
    if (normals) std::copy(nrm.begin(), nrm.end(), normals);
    return STK_OK;
  });
}

static bool positive_finite(const double* v, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!(v[i] > 0) || !std::isfinite(v[i])) return false;
  return true;
}

int stk_set_viscosity(stk_ctx* c, const double* mu_vol, const double* mu_iface, const double* mu_bface) {
  return guard(c, [&]() -> int {
    if (c->p < 0) return fail(c, STK_ERR_INVALID_ARG, "set the discretisation first");
    int64_t nv = count_points(*c, 0), ni = count_points(*c, 1), nbf = count_points(*c, 2);
    if (!mu_vol || (ni && !mu_iface) || (nbf && !mu_bface)) return fail(c, STK_ERR_INVALID_ARG, "null mu");
    if (!positive_finite(mu_vol, nv) || (ni && !positive_finite(mu_iface, ni)) ||
        (nbf && !positive_finite(mu_bface, nbf)))
      return fail(c, STK_ERR_INVALID_ARG, "mu must be finite and positive");
    free_device(*c);
    c->mu_vol.assign(mu_vol, mu_vol + nv);
    c->mu_if.assign(mu_iface, mu_iface + ni);
    c->mu_bf.assign(mu_bface, mu_bface + nbf);
    return STK_OK;
  });
}

int stk_set_density(stk_ctx* c, const double* rho_vol, const double* rho_iface, double delta) {
  return guard(c, [&]() -> int {
    if (c->p < 0) return fail(c, STK_ERR_INVALID_ARG, "set the discretisation first");
    free_device(*c);
    if (delta == 0.0) {
      c->delta = 0.0;
      c->rho_vol.clear();
      c->rho_if.clear();
      return STK_OK;
    }
    if (!(delta > 0) || !rho_vol) return fail(c, STK_ERR_INVALID_ARG, "bad density arguments");
    int64_t nv = count_points(*c, 0), ni = count_points(*c, 1);
    if (ni && !rho_iface) return fail(c, STK_ERR_INVALID_ARG, "null rho_iface");
    if (!positive_finite(rho_vol, nv) || (ni && !positive_finite(rho_iface, ni)))
      return fail(c, STK_ERR_INVALID_ARG, "rho must be finite and positive");
    c->delta = delta;
    c->rho_vol.assign(rho_vol, rho_vol + nv);
    c->rho_if.assign(rho_iface, rho_iface + ni);
    return STK_OK;
  });
}

static void invalidate_graphs(Ctx& c) {
  if (c.graph) cudaGraphExecDestroy(c.graph);
  c.graph = nullptr;
  c.graph_x = c.graph_b = nullptr;
  if (c.cycle_graph) cudaGraphExecDestroy(c.cycle_graph);
  c.cycle_graph = nullptr;
  c.cycle_graph_prec = -1;
  if (c.mgraph) cudaGraphExecDestroy(c.mgraph);
  c.mgraph = nullptr;
  c.mgraph_key[0] = -1;
  if (c.lgraph) cudaGraphExecDestroy(c.lgraph);
  if (c.rgraph) cudaGraphExecDestroy(c.rgraph);
  c.lgraph = c.rgraph = nullptr;
  c.lgraph_x = c.lgraph_b = nullptr;
}

int stk_set_cycle(stk_ctx* c, int nu1, int nu2, int precision) {
  return guard(c, [&]() -> int {
    if (nu1 < 0 || nu2 < 0 || nu1 + nu2 == 0 || precision < 0 || precision > 3)
      return fail(c, STK_ERR_INVALID_ARG, "bad cycle options");
    if (c->ready && precision != c->precision) free_device(*c);
    c->nu1 = nu1;
    c->nu2 = nu2;
    c->precision = precision;
    invalidate_graphs(*c);
    build_persist(*c);
    return STK_OK;
  });
}

int stk_set_colouring(stk_ctx* c, int mode) {
  return guard(c, [&]() -> int {
    if (mode < STK_COLOURS_AUTO || mode > STK_COLOURS_CHECKERBOARD)
      return fail(c, STK_ERR_INVALID_ARG, "bad colouring mode");
    c->colouring = mode;
    return STK_OK;
  });
}

int stk_set_bottom(stk_ctx* c, int64_t max_unknowns) {
  return guard(c, [&]() -> int {
    if (max_unknowns < 0 || max_unknowns > 20000) return fail(c, STK_ERR_INVALID_ARG, "bottom size out of 0..20000");
    c->bottom_max = max_unknowns;
    return STK_OK;
  });
}

int stk_set_clusters(stk_ctx* c, int on) {
  return guard(c, [&]() -> int {
    if (on != 0 && on != 1) return fail(c, STK_ERR_INVALID_ARG, "clusters: 0 or 1");
    c->cluster_req = on;
    return STK_OK;
  });
}

int stk_set_persistent(stk_ctx* c, int max_elements, int ctas_per_sm) {
  return guard(c, [&]() -> int {
    if (max_elements < 0 || ctas_per_sm < 1 || ctas_per_sm > 8)
      return fail(c, STK_ERR_INVALID_ARG, "bad persistent-cycle settings");
    c->persist_max = max_elements;
    c->persist_ctas = ctas_per_sm;
    invalidate_graphs(*c);
    build_persist(*c);
    return STK_OK;
  });
}

int stk_barrier_selftest(stk_ctx* c, int absent, int64_t limit_ticks, int64_t* passed) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (limit_ticks < 1000 || limit_ticks > 4000000000LL) return fail(c, STK_ERR_INVALID_ARG, "bad wait bound");
    const int grid = persist_grid(*c);
    if (absent >= grid) return fail(c, STK_ERR_INVALID_ARG, "no such CTA");
    cudaStream_t st = c->stream;
    unsigned int* cnt = reinterpret_cast<unsigned int*>(c->norm_buf + 1040);
    ck(cudaMemsetAsync(c->gbar, 0, sizeof(GridBarrierWords), st), "memset");
    ck(cudaMemsetAsync(c->dev_err, 0, sizeof(int), st), "memset");
    ck(cudaMemsetAsync(cnt, 0, sizeof(unsigned int), st), "memset");
    ck(launch_barrier_selftest(c->gbar, c->dev_err, (long long)limit_ticks, 4, absent, grid, cnt, st), "selftest");
    c->launches++;
    int err = 0;
    unsigned int n = 0;
    ck(cudaMemcpyAsync(&err, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaMemcpyAsync(&n, cnt, sizeof(unsigned int), cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaStreamSynchronize(st), "sync");
    ck(cudaMemsetAsync(c->dev_err, 0, sizeof(int), st), "memset");
    ck(cudaMemsetAsync(c->gbar, 0, sizeof(GridBarrierWords), st), "memset");
    ck(cudaStreamSynchronize(st), "sync");
    if (passed) *passed = n;
    if (err == kErrBarrierTimeout) return fail(c, STK_ERR_TIMEOUT, "a grid-barrier wait reached its bound");
    if (err != 0) return fail(c, STK_ERR_CUDA, "unexpected error word");
    return STK_OK;
  });
}

int stk_set_cycle_shape(stk_ctx* c, int gamma, int growth, int max_sweeps) {
  return guard(c, [&]() -> int {
    if (gamma < 1 || gamma > 3 || growth < 1 || growth > 4 || max_sweeps < 1 || max_sweeps > 256)
      return fail(c, STK_ERR_INVALID_ARG, "bad cycle shape");
    c->cyc_gamma = gamma;
    c->cyc_growth = growth;
    c->cyc_cap = max_sweeps;
    invalidate_graphs(*c);
    build_persist(*c);
    return STK_OK;
  });
}

// stk_setup for a cut-cell mesh of the embedded circle: the general
// block-sparse hierarchy of cutsetup.cpp on the device.
int setup_cut_device(stk_ctx* c, cudaStream_t st) {
  const double hx = (c->hi[0] - c->lo[0]) / c->n[0], hy = (c->hi[1] - c->lo[1]) / c->n[1];
  if (c->d != 2 || c->n[0] != c->n[1] || c->n[0] < 4 || std::fabs(hx - hy) > 1e-12 * hx)
    return fail(c, STK_ERR_INVALID_ARG, "the embedded circle needs a 2D n x n mesh of square cells, n >= 4");
  for (int i = 0; i < 4; ++i)
    if (c->bc[i] != STK_BC_DIRICHLET) return fail(c, STK_ERR_INVALID_ARG, "cut-cell meshes take Dirichlet sides only");
  if (c->p > 3) return fail(c, STK_ERR_INVALID_ARG, "cut-cell meshes take p = 1..3");
  const size_t nph = c->cut_inside ? 1 : 2;
  if (c->mu_phase.size() != nph) return fail(c, STK_ERR_INVALID_ARG, "set the phase viscosities (stk_set_phases)");
  if (c->cut_delta > 0 && c->rho_phase.size() != nph)
    return fail(c, STK_ERR_INVALID_ARG, "set the phase densities (stk_set_phase_density)");
  if (c->precision != STK_FP64 && c->precision != STK_FP32)
    return fail(c, STK_ERR_INVALID_ARG, "cut-cell levels store FP64 or FP32 blocks");
  if (c->c_intra != 0.0) return fail(c, STK_ERR_INVALID_ARG, "cut-cell meshes take no interior velocity penalty");
  std::string err;
  int rc = setup_cut(*c, err);
  if (rc != STK_OK) return fail(c, rc, err);
  const int L = nlevels(*c);
  if (L < 2) return fail(c, STK_ERR_INVALID_ARG, "mesh too small for a hierarchy");
  c->dev.assign(L, DevLevel());
  try {
    for (int l = 0; l < L - 1; ++l) pack_generic(*c, l, st);
  } catch (const std::runtime_error& e) {
    free_device(*c);
    return fail(c, STK_ERR_SINGULAR_BLOCK, e.what());
  }
  alloc_vectors(*c);
  c->cluster_on = 0;
  setup_bottom(*c);
  c->dev_err = (int*)dalloc(*c, 16);
  ck(cudaMemset(c->dev_err, 0, 16), "memset");
  c->gbar = (GridBarrierWords*)dalloc(*c, 64);
  ck(cudaMemset(c->gbar, 0, 64), "memset");
  ck(cudaStreamSynchronize(st), "setup sync");
  ck(cudaDeviceSynchronize(), "setup sync");
  c->ready = true;
  return STK_OK;
}

int stk_setup(stk_ctx* c, void* stream) {
  return guard(c, [&]() -> int {
    if (c->p < 0) return fail(c, STK_ERR_INVALID_ARG, "set mesh and discretisation first");
    if (c->cut) {
      ck(cudaSetDevice(c->device), "cudaSetDevice");
      free_device(*c);
      return setup_cut_device(c, (cudaStream_t)stream);
    }
    if (c->mu_vol.empty()) return fail(c, STK_ERR_INVALID_ARG, "set the viscosity first");
    if (c->colouring == STK_COLOURS_CHECKERBOARD && (c->gamma != 0 || !c->chi.empty()))
      return fail(c, STK_ERR_INVALID_ARG,
                  "the checkerboard is a valid colouring only for the single-phase standard form");
    ck(cudaSetDevice(c->device), "cudaSetDevice");
    free_device(*c);
    build_pattern(c->d, c->p, c->gamma, !c->chi.empty(), c->pat);
    if (c->pat.T >= kMaxTasks || c->pat.NG >= kMaxGather || c->pat.NO >= kMaxOffsets)
      return fail(c, STK_ERR_INVALID_ARG, "coupling pattern exceeds the library's compiled limits");
    int rc = setup_host(*c);
    if (rc != STK_OK) return rc;
    int L = nlevels(*c);
    if (L < 2) return fail(c, STK_ERR_INVALID_ARG, "mesh too small for a hierarchy (need n >= 4 even)");
    c->dev.assign(L, DevLevel());
    cudaStream_t st = (cudaStream_t)stream;
    try {
      for (int l = 0; l < L - 1; ++l) pack_level(*c, l, st);
    } catch (const std::runtime_error& e) {
      free_device(*c);
      return fail(c, STK_ERR_SINGULAR_BLOCK, e.what());
    }
    alloc_vectors(*c);
    // element clustering of level 0 (2D, p = 1, one phase, a hierarchy below
    // it, every periodic axis with an even number of clusters)
    c->cluster_on = 0;
    if (c->cluster_req && c->d == 2 && c->p == 1 && c->chi.empty() && L >= 3) {
      bool ok = true;
      for (int k = 0; k < c->d; ++k)
        if (c->host[0].n[k] % 2 || (c->bc[2 * k] == STK_BC_PERIODIC && (c->host[0].n[k] / 2) % 2)) ok = false;
      if (ok) {
        build_pattern(c->d, 3, c->gamma, false, c->cpat);
        std::string err;
        if (build_cluster_level(*c, c->host[0], c->pat, c->cpat, c->chost, err) != STK_OK) return fail(c, STK_ERR_INVALID_ARG, err);
        try {
          pack_records(*c, c->chost, c->cpat, c->cdev, false, st);
        } catch (const std::runtime_error& e) {
          free_device(*c);
          return fail(c, STK_ERR_SINGULAR_BLOCK, e.what());
        }
        const int64_t n0 = level_ne(*c, 0) * c->nb;
        for (int v = 0; v < 2; ++v) {
          if (v == 1 && c->precision == STK_FP64) continue;
          const size_t es = v == 0 ? 8 : 4;
          c->cvx[v] = dalloc(*c, n0 * es);
          c->cvb[v] = dalloc(*c, n0 * es);
          c->cvr[v] = dalloc(*c, n0 * es);
          c->ctmp[v] = dalloc(*c, n0 * es);
        }
        c->cluster_on = 1;
      }
    }
    setup_bottom(*c);
    c->dev_err = (int*)dalloc(*c, 16);
    ck(cudaMemset(c->dev_err, 0, 16), "memset");
    static bool prepared[64] = {false};
    if (c->device >= 0 && c->device < 64 && !prepared[c->device]) {
      prepare_pipe_kernels();
      prepare_mrhs_kernels();
      prepare_df_kernels();
      prepared[c->device] = true;
    }
    for (int pr = 0; pr < 3; ++pr)
      if (c->pipe_ctas[pr] <= 0 || c->pipe_stages[pr] <= 0)
        pipe_default_shape(c->pat, pr, &c->pipe_ctas[pr], &c->pipe_stages[pr]);
    std::vector<double> P;
    child_matrices(c->d, c->p, P);
    int s = c->s, nch = 1 << c->d;
    std::vector<double> PT(P.size());
    for (int ch = 0; ch < nch; ++ch)
      for (int a = 0; a < s; ++a)
        for (int b2 = 0; b2 < s; ++b2) PT[((size_t)ch * s + b2) * s + a] = P[((size_t)ch * s + a) * s + b2];
    std::vector<float> P32(P.begin(), P.end()), PT32(PT.begin(), PT.end());
    c->child_P[0] = dalloc(*c, P.size() * 8);
    c->child_PT[0] = dalloc(*c, P.size() * 8);
    c->child_P[1] = dalloc(*c, P.size() * 4);
    c->child_PT[1] = dalloc(*c, P.size() * 4);
    ck(cudaMemcpy(c->child_P[0], P.data(), P.size() * 8, cudaMemcpyHostToDevice), "copy P");
    ck(cudaMemcpy(c->child_PT[0], PT.data(), P.size() * 8, cudaMemcpyHostToDevice), "copy P");
    ck(cudaMemcpy(c->child_P[1], P32.data(), P.size() * 4, cudaMemcpyHostToDevice), "copy P");
    ck(cudaMemcpy(c->child_PT[1], PT32.data(), P.size() * 4, cudaMemcpyHostToDevice), "copy P");
    c->gbar = (GridBarrierWords*)dalloc(*c, 64);
    ck(cudaMemset(c->gbar, 0, 64), "memset");
    ck(cudaStreamSynchronize(st), "setup sync");
    ck(cudaDeviceSynchronize(), "setup sync");
    c->ready = true;
    build_persist(*c);
    return STK_OK;
  });
}

int stk_get_sizes(stk_ctx* c, int* nl, int64_t* ne, int* nb, int* snapped) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (nl) *nl = nlevels(*c);
    if (ne)
      for (int l = 0; l < nlevels(*c); ++l) ne[l] = level_ne(*c, l);
    if (nb) *nb = c->nb;
    if (snapped) *snapped = c->n_snapped;
    return STK_OK;
  });
}

int stk_get_info(stk_ctx* c, int what, int64_t* value) {
  return guard(c, [&]() -> int {
    if (!value) return fail(c, STK_ERR_INVALID_ARG, "null output");
    switch (what) {
      case STK_INFO_BOTTOM_SOLVER:
        if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
        *value = c->bottom_solver;
        return STK_OK;
      case STK_INFO_BOTTOM_UNKNOWNS:
        if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
        *value = c->nbot;
        return STK_OK;
      case STK_INFO_COLOURS:
        if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
        *value = nlevels(*c) > 1 ? c->dev[0].ncolour : 0;
        return STK_OK;
      case STK_INFO_CLUSTERS:
        if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
        *value = c->cluster_on;
        return STK_OK;
      case STK_INFO_DEVICE_BYTES:
        *value = c->device_bytes;
        return STK_OK;
      case STK_INFO_COUPLING_BLOCKS:
        if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
        *value = c->cut ? (int64_t)c->host[0].tnbr.size() : (int64_t)c->host[0].ne * c->pat.T;
        return STK_OK;
      default:
        return fail(c, STK_ERR_INVALID_ARG, "unknown info key");
    }
  });
}

int stk_get_block(stk_ctx* c, int level, int64_t i, int64_t j, double* out) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (level < 0 || level >= nlevels(*c) || !out) return fail(c, STK_ERR_INVALID_ARG, "bad level");
    const HostLevel& H = c->host[level];
    if (i < 0 || j < 0 || i >= H.ne || j >= H.ne) return fail(c, STK_ERR_INVALID_ARG, "bad element");
    int nb = c->nb, s = c->s, ss = s * s;
    std::fill(out, out + (size_t)nb * nb, 0.0);
    if (i == j) std::copy(&H.D[(size_t)i * nb * nb], &H.D[(size_t)(i + 1) * nb * nb], out);
    if (c->cut) {
      for (int t = H.tptr[i]; t < H.tptr[i + 1]; ++t) {
        if (H.tnbr[t] != j) continue;
        const int rv = H.tvar[t] / 4, cv = H.tvar[t] % 4;
        for (int a = 0; a < s; ++a)
          for (int b = 0; b < s; ++b) out[(size_t)(rv * s + a) * nb + cv * s + b] += H.C[(size_t)t * ss + a * s + b];
      }
      return STK_OK;
    }
    for (int t = 0; t < c->pat.T; ++t) {
      if (H.nbr[(size_t)i * c->pat.NO + c->pat.task_o[t]] != j) continue;
      int rv = c->pat.task_rv[t], cv = c->pat.task_cv[t];
      for (int a = 0; a < s; ++a)
        for (int b = 0; b < s; ++b)
          out[(size_t)(rv * s + a) * nb + cv * s + b] += H.C[((size_t)i * c->pat.T + t) * ss + a * s + b];
    }
    return STK_OK;
  });
}

int stk_assemble_rhs(stk_ctx* c, const double* f_vol, const double* bdata, double* b) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (!f_vol || !b) return fail(c, STK_ERR_INVALID_ARG, "null argument");
    if (c->cut) return fail(c, STK_ERR_INVALID_ARG, "cut-cell meshes take stk_assemble_rhs2 (interface data)");
    if (count_points(*c, 2) > 0 && !bdata) return fail(c, STK_ERR_INVALID_ARG, "null boundary data");
    return assemble_rhs_host(*c, f_vol, bdata, b);
  });
}

int stk_residual(stk_ctx* c, const double* x, const double* b, double* r, double* norm_out, void* stream) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (!x || !b || !r) return fail(c, STK_ERR_INVALID_ARG, "null vector");
    cudaStream_t st = (cudaStream_t)stream;
    enqueue_residual64(*c, x, b, r, st);
    if (norm_out) {
      enqueue_norm(*c, r, st);
      ck(cudaStreamSynchronize(st), "sync");
      *norm_out = std::sqrt(c->norm_host[0]);
    }
    return STK_OK;
  });
}

int stk_gs_colour(stk_ctx* c, int level, int colour, double* x, const double* b, void* stream) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (level < 0 || level >= nlevels(*c) - 1) return fail(c, STK_ERR_INVALID_ARG, "bad level");
    if (colour < 0 || colour >= c->dev[level].ncolour || !x || !b) return fail(c, STK_ERR_INVALID_ARG, "bad colour");
    DevLevel& D = c->dev[level];
    int n = D.cstart[colour + 1] - D.cstart[colour];
    ck(run_element(*c, level, STK_FP64, MODE_GS, D.cstart[colour], n, D.inv[0], b, x, nullptr,
                   (cudaStream_t)stream),
       "gs colour launch");
    c->launches++;
    return STK_OK;
  });
}

static bool have_precision(const Ctx& c, int precision) {
  return precision == STK_FP64 || (precision == c.precision && precision > 0 && precision <= 3);
}

int stk_gs_colour_ex(stk_ctx* c, int level, int colour, int precision, void* x, const void* b,
                     void* stream) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (level < 0 || level >= nlevels(*c) - 1) return fail(c, STK_ERR_INVALID_ARG, "bad level");
    if (colour < 0 || colour >= c->dev[level].ncolour || !x || !b) return fail(c, STK_ERR_INVALID_ARG, "bad colour");
    if (!have_precision(*c, precision)) return fail(c, STK_ERR_INVALID_ARG, "precision not set up");
    DevLevel& D = c->dev[level];
    int n = D.cstart[colour + 1] - D.cstart[colour];
    ck(run_element(*c, level, precision, MODE_GS, D.cstart[colour], n, D.inv[precision], b, x, nullptr,
                   (cudaStream_t)stream),
       "gs colour launch");
    c->launches++;
    return STK_OK;
  });
}

int stk_residual_ex(stk_ctx* c, int level, int precision, const void* x, const void* b, void* r,
                    void* stream) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (level < 0 || level >= nlevels(*c) - 1) return fail(c, STK_ERR_INVALID_ARG, "bad level");
    if (!x || !b || !r) return fail(c, STK_ERR_INVALID_ARG, "null vector");
    if (!have_precision(*c, precision)) return fail(c, STK_ERR_INVALID_ARG, "precision not set up");
    DevLevel& D = c->dev[level];
    ck(run_element(*c, level, precision, MODE_RESID, 0, D.ne, D.dia[precision], b, (void*)x, r,
                   (cudaStream_t)stream),
       "residual launch");
    c->launches++;
    return STK_OK;
  });
}

int stk_vcycle(stk_ctx* c, double* x, const double* b, void* stream) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (!x || !b) return fail(c, STK_ERR_INVALID_ARG, "null vector");
    enqueue_cycle(*c, STK_FP64, 0, x, b, (cudaStream_t)stream);
    return STK_OK;
  });
}

int stk_restrict(stk_ctx* c, int level, const double* r, double* rc, void* stream) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (level < 0 || level >= nlevels(*c) - 1 || !r || !rc) return fail(c, STK_ERR_INVALID_ARG, "bad args");
    DevLevel& D = c->dev[level];
    DevLevel& Dc = c->dev[level + 1];
    ck(D.gen ? launch_gen_restrict(1, Dc.ne, c->s, c->nb, D.gcptr, D.gclist, D.gI[0], r, rc, (cudaStream_t)stream)
             : launch_restrict(1, c->d, c->s, c->nb, Dc.n, D.n, Dc.ne, c->child_P[0], r, rc, (cudaStream_t)stream),
       "restrict");
    c->launches++;
    return STK_OK;
  });
}

int stk_prolong(stk_ctx* c, int level, const double* xc, double* x, void* stream) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (level < 0 || level >= nlevels(*c) - 1 || !xc || !x) return fail(c, STK_ERR_INVALID_ARG, "bad args");
    DevLevel& D = c->dev[level];
    DevLevel& Dc = c->dev[level + 1];
    ck(D.gen ? launch_gen_prolong(1, D.ne, c->s, c->nb, D.gparent, D.gI[0], xc, x, (cudaStream_t)stream)
             : launch_prolong(1, c->d, c->s, c->nb, D.n, Dc.n, Dc.ne, c->child_PT[0], xc, x, (cudaStream_t)stream),
       "prolong");
    c->launches++;
    return STK_OK;
  });
}

int stk_bottom_solve(stk_ctx* c, const double* b, double* x, void* stream) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (!b || !x) return fail(c, STK_ERR_INVALID_ARG, "null vector");
    ck(launch_bottom(1, c->nbot, c->bottom_pinv, b, x, (cudaStream_t)stream), "bottom");
    c->launches++;
    return STK_OK;
  });
}

int stk_solve(stk_ctx* c, double* x, const double* b, double rtol, int maxit, int* iters_out, double* hist,
              void* stream) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (!x || !b || maxit < 0 || !(rtol > 0)) return fail(c, STK_ERR_INVALID_ARG, "bad solve arguments");
    cudaStream_t user = (cudaStream_t)stream;
    ck(cudaStreamSynchronize(user), "sync caller stream");
    cudaStream_t st = c->stream;
    ck(cudaMemsetAsync(c->dev_err, 0, sizeof(int), st), "clear error word");
    // ||b||, and ||x|| to recognise a zero first guess
    enqueue_norm(*c, b, st);
    ck(cudaStreamSynchronize(st), "sync");
    const double bnorm_true = std::sqrt(c->norm_host[0]);
    double bnorm = bnorm_true == 0.0 ? 1.0 : bnorm_true;
    enqueue_norm(*c, x, st);
    ck(cudaStreamSynchronize(st), "sync");
    double rnorm;
    if (c->norm_host[0] == 0.0) {
      // x = 0: b - A x is b itself, exactly (no pass over the FP64 records)
      ck(cudaMemcpyAsync(c->r64, b, (size_t)level_ne(*c, 0) * c->nb * sizeof(double), cudaMemcpyDeviceToDevice, st),
         "r = b");
      rnorm = bnorm_true;
    } else {
      enqueue_residual64(*c, x, b, c->r64, st);
      enqueue_norm(*c, c->r64, st);
      ck(cudaStreamSynchronize(st), "sync");
      rnorm = std::sqrt(c->norm_host[0]);
    }
    double rel = rnorm / bnorm, rel0 = rel;
    if (hist) hist[0] = rel;
    int it = 0;
    const bool learned = c->learn_on && c->lW1 && c->precision != STK_FP64;
    if (learned && c->solver != 0)
      return fail(c, STK_ERR_INVALID_ARG,
                  "the learned correction is judged on the outer residual of every cycle: use outer method 0");
    if (c->solver >= 1) {
      try {
        it = fgmres(*c, x, b, rtol, maxit, hist, bnorm, rel, st);
      } catch (const Timeout&) {
        return fail(c, STK_ERR_TIMEOUT, "a kernel's bounded wait for its records expired");
      }
      if (iters_out) *iters_out = it;
      if (!std::isfinite(rel) || rel > 1e6 * rel0) return fail(c, STK_ERR_DIVERGED, "outer iteration diverged");
      return STK_OK;
    }
    // Capture one outer iteration as a CUDA graph (re-captured when the
    // caller's vectors or the precision change).
    if (!c->graph || c->graph_x != x || c->graph_b != b || c->graph_prec != c->precision) {
      if (c->graph) cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
      cudaGraph_t g;
      int64_t before = c->launches;
      ck(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
      try {
        enqueue_iteration(*c, x, b, st);
      } catch (...) {
        cudaStreamEndCapture(st, &g);
        throw;
      }
      ck(cudaStreamEndCapture(st, &g), "end capture");
      ck(cudaGraphInstantiate(&c->graph, g, 0), "graph instantiate");
      cudaGraphDestroy(g);
      c->graph_kernels = c->launches - before;
      c->launches = before;
      c->graph_x = x;
      c->graph_b = b;
      c->graph_prec = c->precision;
    }
    if (learned && (!c->lgraph || c->lgraph_x != x || c->lgraph_b != b)) {
      if (c->lgraph) cudaGraphExecDestroy(c->lgraph);
      if (c->rgraph) cudaGraphExecDestroy(c->rgraph);
      c->lgraph = c->rgraph = nullptr;
      c->lgraph = capture_graph(*c, st, [&]() { enqueue_learned_iteration(*c, x, b, st); }, &c->lgraph_kernels);
      c->rgraph = capture_graph(*c, st, [&]() { enqueue_undo(*c, x, b, st); }, &c->rgraph_kernels);
      c->lgraph_x = x;
      c->lgraph_b = b;
    }
    // Learned correction: kappa from the first two (plain) iterations, then
    // each correction kept only if ||r_new|| < kappa ||r_old||; two
    // consecutive rejections switch it off for the rest of the solve.
    c->l_hist.clear();
    c->l_ratio.clear();
    c->l_kappa = 0.0;
    bool active = learned;
    int consecutive = 0;
    auto run = [&](cudaGraphExec_t g, int64_t kernels) -> int {
      ck(cudaGraphLaunch(g, st), "graph launch");
      c->launches += kernels;
      ck(cudaStreamSynchronize(st), "sync");
      if (reinterpret_cast<int*>(c->norm_host + 1)[0] != 0)
        return fail(c, STK_ERR_TIMEOUT, "a kernel's bounded wait for its records expired");
      return STK_OK;
    };
    while (rel > rtol && it < maxit) {
      const double rel_old = rel;
      if (active && it >= 2) {
        int rc2 = run(c->lgraph, c->lgraph_kernels);
        if (rc2 != STK_OK) return rc2;
        const double rel_new = std::sqrt(c->norm_host[0]) / bnorm;
        const double ratio = rel_new / (c->l_kappa * rel_old);
        c->l_ratio.push_back(ratio);
        if (ratio < 1.0) {
          c->l_hist.push_back(1);
          c->l_acc++;
          consecutive = 0;
        } else {
          rc2 = run(c->rgraph, c->rgraph_kernels);
          if (rc2 != STK_OK) return rc2;
          c->l_hist.push_back(0);
          c->l_rej++;
          if (++consecutive >= 2) active = false;
        }
      } else {
        int rc2 = run(c->graph, c->graph_kernels);
        if (rc2 != STK_OK) return rc2;
        c->l_hist.push_back(-1);
        c->l_ratio.push_back(0.0);
      }
      rel = std::sqrt(c->norm_host[0]) / bnorm;
      ++it;
      if (it == 2) c->l_kappa = std::sqrt(rel / rel0);
      if (hist) hist[it] = rel;
      if (!std::isfinite(rel) || rel > 1e6 * rel0) {
        if (iters_out) *iters_out = it;
        return fail(c, STK_ERR_DIVERGED, "outer iteration diverged");
      }
    }
    if (iters_out) *iters_out = it;
    return STK_OK;
  });
}

int stk_set_launch_overlap(stk_ctx* c, int on) {
  return guard(c, [&]() -> int {
    if (on != 0 && on != 1) return fail(c, STK_ERR_INVALID_ARG, "launch overlap is 0 or 1");
    c->launch_overlap = on;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    c->graph_x = c->graph_b = nullptr;
    if (c->cycle_graph) cudaGraphExecDestroy(c->cycle_graph);
    c->cycle_graph = nullptr;
    c->cycle_graph_prec = -1;
    return STK_OK;
  });
}

int stk_set_tuning(stk_ctx* c, int variant, int precision, int ctas_per_sm, int stages) {
  return guard(c, [&]() -> int {
    if (variant < 0 || variant > 3 || precision < 0 || precision > 3 || ctas_per_sm < 0 || ctas_per_sm > 32 ||
        stages < 0 || stages > 16)
      return fail(c, STK_ERR_INVALID_ARG, "bad tuning options");
    c->variant_of[precision] = variant;
    if (variant == 2 && ctas_per_sm > 0) c->warp_ctas[precision] = ctas_per_sm;
    if (variant == 3) {
      if (ctas_per_sm == 3 || ctas_per_sm > 4)
        return fail(c, STK_ERR_INVALID_ARG, "variant 3 takes 1, 2 or 4 warps per element");
      c->ring_warps[precision] = ctas_per_sm > 0 ? ctas_per_sm : 2;
    }
    if (variant == 1 && ctas_per_sm > 0 && stages > 0) {
      c->pipe_ctas[precision] = ctas_per_sm;
      c->pipe_stages[precision] = stages;
    } else if (c->ready) {
      pipe_default_shape(c->pat, precision, &c->pipe_ctas[precision], &c->pipe_stages[precision]);
    }
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    c->graph_x = c->graph_b = nullptr;
    if (c->cycle_graph) cudaGraphExecDestroy(c->cycle_graph);
    c->cycle_graph = nullptr;
    c->cycle_graph_prec = -1;
    return STK_OK;
  });
}

int stk_set_wide_launch(stk_ctx* c, int max_positions) {
  return guard(c, [&]() -> int {
    if (max_positions < 0) return fail(c, STK_ERR_INVALID_ARG, "max_positions must be >= 0");
    c->wide_max = max_positions;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    c->graph_x = c->graph_b = nullptr;
    if (c->cycle_graph) cudaGraphExecDestroy(c->cycle_graph);
    c->cycle_graph = nullptr;
    c->cycle_graph_prec = -1;
    if (c->mgraph) cudaGraphExecDestroy(c->mgraph);   // the eight-RHS tensor kernels use the same limit
    c->mgraph = nullptr;
    c->mgraph_key[0] = -1;
    return STK_OK;
  });
}

// Autotuner (no counterpart in the paper; the launch-shape choice of a10):
// times one finest-level colour step for each candidate shape on this
// context's own records, keeps the fastest, then finds the launch size below
// which the one-CTA-per-element kernel beats it, level by level.
int stk_autotune(stk_ctx* c, int* choice, double* best_ms, void* stream) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (c->cut) return fail(c, STK_ERR_INVALID_ARG, "not available on cut-cell meshes");
    cudaStream_t st = (cudaStream_t)stream;
    const int L = nlevels(*c);
    for (int l = 0; l < L - 1; ++l)
      for (int v = 0; v < 2; ++v) {
        DevLevel& D = c->dev[l];
        const size_t es = v == 0 ? 8 : 4;
        if (D.vx[v]) ck(cudaMemsetAsync(D.vx[v], 0, (size_t)D.ne * c->nb * es, st), "memset");
        if (D.vb[v]) ck(cudaMemsetAsync(D.vb[v], 0, (size_t)D.ne * c->nb * es, st), "memset");
      }
    cudaEvent_t e0, e1;
    ck(cudaEventCreate(&e0), "event");
    ck(cudaEventCreate(&e1), "event");
    // Mean time (ms) of one colour-0 step on level l in precision prec: `reps`
    // steps captured in a CUDA graph on the library's own stream and replayed,
    // so that host launch overhead does not hide the kernels' own durations.
    cudaStream_t ts = c->stream;
    ck(cudaStreamSynchronize(st), "sync");
    // The steps cycle through the level's colours, as a sweep does, so that
    // a level whose one colour would fit in L2 is not timed from L2.
    auto time_step = [&](int l, int prec, int reps) -> double {
      DevLevel& D = c->dev[l];
      const int vi = prec == STK_FP64 ? 0 : 1;
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      ck(cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal), "capture");
      for (int i = 0; i < reps; ++i) {
        const int col = i % D.ncolour;
        const int n = D.cstart[col + 1] - D.cstart[col];
        cudaError_t e = run_element(*c, l, prec, MODE_GS, D.cstart[col], n, D.inv[prec], D.vb[vi], D.vx[vi], nullptr,
                                    ts);
        if (e != cudaSuccess) {
          cudaStreamEndCapture(ts, &graph);
          if (graph) cudaGraphDestroy(graph);
          ck(e, "tune launch");
        }
      }
      ck(cudaStreamEndCapture(ts, &graph), "capture");
      ck(cudaGraphInstantiate(&exec, graph, 0), "instantiate");
      ck(cudaGraphLaunch(exec, ts), "graph");
      ck(cudaEventRecord(e0, ts), "event");
      ck(cudaGraphLaunch(exec, ts), "graph");
      ck(cudaEventRecord(e1, ts), "event");
      ck(cudaEventSynchronize(e1), "event");
      float ms = 0;
      ck(cudaEventElapsedTime(&ms, e0, e1), "event");
      cudaGraphExecDestroy(exec);
      cudaGraphDestroy(graph);
      return (double)ms / reps;
    };
    c->wide_max = 0;
    const int precs[2] = {c->precision, STK_FP64};
    double best[2] = {0, 0};
    for (int pi = 0; pi < (c->precision == STK_FP64 ? 1 : 2); ++pi) {
      const int prec = precs[pi];
      // warp-per-element kernel: CTAs of 8 warps per SM
      double t2 = 1e300;
      int bc = c->warp_ctas[prec];
      c->variant_of[prec] = 2;
      for (int ctas : {2, 3, 4, 6, 8}) {
        c->warp_ctas[prec] = ctas;
        const double t = time_step(0, prec, 10);
        if (t < t2) {
          t2 = t;
          bc = ctas;
        }
      }
      c->warp_ctas[prec] = bc;
      // one CTA per element with direct loads (not for scaled FP16 records)
      double t0 = 1e300;
      if (prec != STK_FP16) {
        c->variant_of[prec] = 0;
        t0 = time_step(0, prec, 10);
      }
      // 16-bit records: the warp kernel with the next element staged (falls
      // back to the plain warp kernel where the shape does not fit)
      double t3 = 1e300;
      if (prec == STK_FP16 || prec == STK_BF16) {
        c->variant_of[prec] = 3;
        int bw = 2;
        for (int w : {1, 2}) {
          c->ring_warps[prec] = w;
          const double t = time_step(0, prec, 10);
          if (t < t3) {
            t3 = t;
            bw = w;
          }
        }
        c->ring_warps[prec] = bw;
      }
      c->variant_of[prec] = t3 < std::min(t0, t2) ? 3 : (t0 < t2 ? 0 : 2);
      best[pi] = std::min(std::min(t0, t2), t3);
    }
    // FGMRES matvec of a low-precision cycle: FP32-unit double-float kernel or
    // the FP64 residual kernel, whichever is faster over the whole level 0.
    if (c->precision != STK_FP64 && c->dev[0].cpl_lo) {
      DevLevel& D0 = c->dev[0];
      auto time_matvec = [&](bool df) -> double {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        ck(cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal), "capture");
        for (int i = 0; i < 3; ++i) {
          cudaError_t e = df ? launch_element_df(c->pat, 0, D0.ne, D0.perm, D0.nbr, D0.cpl[STK_FP32], D0.cpl_lo,
                                                 D0.dia[STK_FP32], D0.dia_lo, (const float*)D0.vx[1],
                                                 (double*)D0.vr[0], c->warp_ctas[STK_FP32], ts)
                             : run_element(*c, 0, STK_FP64, MODE_RESID, 0, D0.ne, D0.dia[0], D0.vb[0], D0.vx[0],
                                           D0.vr[0], ts);
          if (e != cudaSuccess) {
            cudaStreamEndCapture(ts, &graph);
            if (graph) cudaGraphDestroy(graph);
            ck(e, "tune matvec");
          }
        }
        ck(cudaStreamEndCapture(ts, &graph), "capture");
        ck(cudaGraphInstantiate(&exec, graph, 0), "instantiate");
        ck(cudaGraphLaunch(exec, ts), "graph");
        ck(cudaEventRecord(e0, ts), "event");
        ck(cudaGraphLaunch(exec, ts), "graph");
        ck(cudaEventRecord(e1, ts), "event");
        ck(cudaEventSynchronize(e1), "event");
        float ms = 0;
        ck(cudaEventElapsedTime(&ms, e0, e1), "event");
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return (double)ms / 3;
      };
      c->df_matvec = time_matvec(true) < time_matvec(false) ? 1 : 0;
    }
    // Latency kernel: time both kernels on every smoothing level's colour
    // step and keep the threshold (0 or one level's colour size) with the
    // least total time over the levels.
    std::vector<int> nl(L - 1);
    std::vector<double> t_cfg(L - 1), t_wide(L - 1);
    for (int l = 0; l < L - 1; ++l) {
      DevLevel& D = c->dev[l];
      nl[l] = 0;
      for (int col = 0; col < D.ncolour; ++col) nl[l] = std::max(nl[l], D.cstart[col + 1] - D.cstart[col]);
      c->wide_max = 0;
      t_cfg[l] = time_step(l, c->precision, 20);
      c->wide_max = nl[l];
      t_wide[l] = time_step(l, c->precision, 20);
    }
    int wide = 0;
    double best_total = 1e300;
    std::vector<int> cand(nl);
    cand.push_back(0);
    for (int thr : cand) {
      double tot = 0;
      for (int l = 0; l < L - 1; ++l) tot += nl[l] <= thr ? t_wide[l] : t_cfg[l];
      if (tot < best_total) {
        best_total = tot;
        wide = thr;
      }
    }
    c->wide_max = wide;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int l = 0; l < L - 1; ++l)
      for (int v = 0; v < 2; ++v) {
        DevLevel& D = c->dev[l];
        const size_t es = v == 0 ? 8 : 4;
        if (D.vx[v]) ck(cudaMemsetAsync(D.vx[v], 0, (size_t)D.ne * c->nb * es, st), "memset");
      }
    ck(cudaStreamSynchronize(st), "sync");
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    c->graph_x = c->graph_b = nullptr;
    if (c->cycle_graph) cudaGraphExecDestroy(c->cycle_graph);
    c->cycle_graph = nullptr;
    c->cycle_graph_prec = -1;
    if (choice) {
      choice[0] = c->variant_of[c->precision];
      choice[1] = c->variant_of[c->precision] == 3 ? c->ring_warps[c->precision] : c->warp_ctas[c->precision];
      choice[2] = c->variant_of[STK_FP64];
      choice[3] = c->warp_ctas[STK_FP64];
      choice[4] = c->wide_max;
      choice[5] = c->df_matvec;
    }
    if (best_ms) {
      best_ms[0] = best[0];
      best_ms[1] = c->precision == STK_FP64 ? best[0] : best[1];
    }
    return STK_OK;
  });
}

int stk_set_df_matvec(stk_ctx* c, int on) {
  return guard(c, [&]() -> int {
    c->df_matvec = on ? 1 : 0;
    return STK_OK;
  });
}

int stk_set_mrhs_tensor(stk_ctx* c, int on) {
  return guard(c, [&]() -> int {
    c->mrhs_tensor = on ? 1 : 0;
    if (c->mgraph) cudaGraphExecDestroy(c->mgraph);
    c->mgraph = nullptr;
    c->mgraph_key[0] = -1;
    return STK_OK;
  });
}

int stk_gmres_rho(stk_ctx* c, const double* x0, double reduction, int maxit, double* rho_out, int* iters_out,
                  double* hist, double* hess, void* stream) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (!x0 || !rho_out || !(reduction > 0 && reduction < 1) || maxit < 1 || maxit > 100)
      return fail(c, STK_ERR_INVALID_ARG, "bad arguments (reduction in (0,1), maxit 1..100)");
    ck(cudaStreamSynchronize((cudaStream_t)stream), "sync caller stream");
    if (hess) std::fill(hess, hess + (size_t)(maxit + 1) * maxit, 0.0);
    double rho = 0;
    int n = 0;
    try {
      n = gmres_rho(*c, x0, reduction, maxit, hist, hess, rho, c->stream);
    } catch (const Timeout&) {
      return fail(c, STK_ERR_TIMEOUT, "a kernel's bounded wait for its records expired");
    }
    *rho_out = rho;
    if (iters_out) *iters_out = n;
    if (!std::isfinite(rho)) return fail(c, STK_ERR_DIVERGED, "GMRES residual not finite");
    return STK_OK;
  });
}

int stk_set_solver(stk_ctx* c, int method, int restart) {
  return guard(c, [&]() -> int {
    if (method < 0 || method > 2 || restart < 1 || restart > 100)
      return fail(c, STK_ERR_INVALID_ARG, "bad solver options (method 0/1/2, restart 1..100)");
    c->solver = method;
    if (restart != c->restart) {
      c->restart = restart;
      c->kV = nullptr;   // re-sized on the next solve (old buffers stay owned until destroy)
      c->kcap = 0;
    }
    return STK_OK;
  });
}

int stk_solve_multi(stk_ctx* c, double* X, const double* B, int nrhs, double rtol, int maxit, int inner,
                    int* iters_out, double* hist, void* stream) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (c->cut) return fail(c, STK_ERR_INVALID_ARG, "not available on cut-cell meshes");
    if (!X || !B || nrhs < 1 || nrhs > 8 || maxit < 0 || inner < 1 || inner > 16 || !(rtol > 0))
      return fail(c, STK_ERR_INVALID_ARG, "bad multi-rhs arguments (1 <= nrhs <= 8, 1 <= inner <= 16)");
    if (c->precision == STK_FP16)
      return fail(c, STK_ERR_INVALID_ARG, "several right-hand sides take FP64, FP32 or BF16 blocks");
    int nr = nrhs <= 4 ? 4 : 8;
    cudaStream_t user = (cudaStream_t)stream;
    ck(cudaStreamSynchronize(user), "sync caller stream");
    cudaStream_t st = c->stream;
    ensure_mrhs(*c, nr);
    int64_t m = level_ne(*c, 0) * c->nb;
    ck(launch_interleave(0, m, nr, nrhs, 1, c->mB, B, st), "interleave");
    ck(launch_interleave(0, m, nr, nrhs, 1, c->mX, X, st), "interleave");
    c->launches += 2;
    ck(launch_sumsq_mr(m, nr, c->mB, c->mPart, c->mNorm, st), "norms");
    c->launches += 2;
    ck(cudaMemcpyAsync(c->norm_host, c->mNorm, nr * 8, cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaStreamSynchronize(st), "sync");
    std::vector<double> bn(nr), rel(nr);
    for (int q = 0; q < nrhs; ++q) bn[q] = c->norm_host[q] > 0 ? std::sqrt(c->norm_host[q]) : 1.0;
    DevLevel& D0 = c->dev[0];
    ck(launch_element_mrhs(c->pat, STK_FP64, nr, MODE_RESID, 0, D0.ne, D0.perm, D0.nbr, D0.cpl[0], D0.dia[0], c->mB,
                           c->mX, c->mR, st, c->mrhs_tensor, c->wide_max),
       "residual64");
    ck(launch_sumsq_mr(m, nr, c->mR, c->mPart, c->mNorm, st), "norms");
    c->launches += 3;
    ck(cudaMemcpyAsync(c->norm_host, c->mNorm, nr * 8, cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaStreamSynchronize(st), "sync");
    auto check = [&](int it) {
      bool done = true;
      for (int q = 0; q < nrhs; ++q) {
        rel[q] = std::sqrt(c->norm_host[q]) / bn[q];
        if (hist) hist[(size_t)it * nrhs + q] = rel[q];
        if (!(rel[q] <= rtol)) done = false;
      }
      return done;
    };
    std::vector<double> rel0;
    bool done = check(0);
    rel0 = rel;
    if (c->solver >= 1) {
      // flexible GMRES in lockstep over the right-hand sides
      int it = done ? 0 : fgmres_mr(*c, nr, nrhs, rtol, maxit, hist, bn, rel, st);
      ck(launch_interleave(0, m, nr, nrhs, 0, X, c->mX, st), "deinterleave");
      c->launches++;
      ck(cudaStreamSynchronize(st), "sync");
      if (iters_out) *iters_out = it;
      for (int q = 0; q < nrhs; ++q)
        if (!std::isfinite(rel[q]) || rel[q] > 1e6 * rel0[q]) return fail(c, STK_ERR_DIVERGED, "outer iteration diverged");
      return STK_OK;
    }
    int key[3] = {nr, inner, c->precision};
    if (!c->mgraph || c->mgraph_key[0] != key[0] || c->mgraph_key[1] != key[1] || c->mgraph_key[2] != key[2]) {
      if (c->mgraph) cudaGraphExecDestroy(c->mgraph);
      c->mgraph = nullptr;
      cudaGraph_t g;
      int64_t before = c->launches;
      ck(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
      try {
        enqueue_mr_iteration(*c, nr, inner, st);
      } catch (...) {
        cudaStreamEndCapture(st, &g);
        c->launches = before;
        throw;
      }
      ck(cudaStreamEndCapture(st, &g), "end capture");
      ck(cudaGraphInstantiate(&c->mgraph, g, 0), "graph instantiate");
      cudaGraphDestroy(g);
      c->mgraph_kernels = c->launches - before;
      c->launches = before;
      for (int i = 0; i < 3; ++i) c->mgraph_key[i] = key[i];
    }
    int it = 0;
    while (!done && it < maxit) {
      ck(cudaGraphLaunch(c->mgraph, st), "graph launch");
      c->launches += c->mgraph_kernels;
      ck(cudaStreamSynchronize(st), "sync");
      ++it;
      done = check(it);
      for (int q = 0; q < nrhs; ++q)
        if (!std::isfinite(rel[q]) || rel[q] > 1e6 * rel0[q]) {
          if (iters_out) *iters_out = it;
          return fail(c, STK_ERR_DIVERGED, "outer iteration diverged");
        }
    }
    ck(launch_interleave(0, m, nr, nrhs, 0, X, c->mX, st), "deinterleave");
    c->launches++;
    ck(cudaStreamSynchronize(st), "sync");
    if (iters_out) *iters_out = it;
    return STK_OK;
  });
}

// splitmix-style deterministic weight initialisation, uniform(-a, a)
static void init_uniform(std::vector<float>& w, uint64_t seed, float a) {
  uint64_t z = seed;
  for (auto& v : w) {
    z += 0x9E3779B97F4A7C15ULL;
    uint64_t t = z;
    t = (t ^ (t >> 30)) * 0xBF58476D1CE4E5B9ULL;
    t = (t ^ (t >> 27)) * 0x94D049BB133111EBULL;
    t ^= t >> 31;
    v = a * (float)((double)(t >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
  }
}

int stk_learn_setup(stk_ctx* c, int hidden, uint64_t seed) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (c->precision == STK_FP64) return fail(c, STK_ERR_INVALID_ARG, "the learned smoother runs in FP32/BF16 cycles");
    if (hidden < 8 || hidden > 512) return fail(c, STK_ERR_INVALID_ARG, "hidden width must be in 8..512");
    const int nb = c->nb, ne = c->dev[0].ne;
    c->l_in = (1 + 2 * c->d) * nb;
    c->l_ldf = (c->l_in + 3) / 4 * 4;
    c->l_hid = hidden;
    int64_t n1 = (int64_t)c->l_in * hidden, n2 = hidden, n3 = (int64_t)hidden * nb, n4 = nb;
    c->l_nparam = n1 + n2 + n3 + n4;
    float* wbase = (float*)dalloc(*c, c->l_nparam * 4);
    c->lW1 = wbase;
    c->lb1 = wbase + n1;
    c->lW2 = c->lb1 + n2;
    c->lb2 = c->lW2 + n3;
    c->lgrad = (float*)dalloc(*c, c->l_nparam * 4);
    c->lm = (float*)dalloc(*c, c->l_nparam * 4);
    c->lv = (float*)dalloc(*c, c->l_nparam * 4);
    ck(cudaMemset(c->lm, 0, c->l_nparam * 4), "memset");
    ck(cudaMemset(c->lv, 0, c->l_nparam * 4), "memset");
    std::vector<float> w(c->l_nparam, 0.f);
    std::vector<float> w1(n1), w2(n3);
    init_uniform(w1, seed, 1.f / std::sqrt((float)c->l_in));
    init_uniform(w2, seed ^ 0x5DEECE66DULL, 0.1f / std::sqrt((float)hidden));   // start near zero correction
    std::copy(w1.begin(), w1.end(), w.begin());
    std::copy(w2.begin(), w2.end(), w.begin() + n1 + n2);
    ck(cudaMemcpy(wbase, w.data(), c->l_nparam * 4, cudaMemcpyHostToDevice), "copy weights");
    c->l_adam_t = 0;
    c->l_ndev = (int*)dalloc(*c, 16);
    ck(cudaMemcpy(c->l_ndev, c->host[0].n, 3 * sizeof(int), cudaMemcpyHostToDevice), "copy n");
    if (c->cut) {
      // neighbours across the anchor cell's faces in the element's phase
      std::vector<int> nbr;
      std::vector<double> ctr;
      cut_face_neighbours(*c, nbr, ctr);
      c->l_no = 4;
      c->l_nbr = (int*)dalloc(*c, nbr.size() * 4);
      ck(cudaMemcpy(c->l_nbr, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice), "copy nbr");
      c->l_ctr = (double*)dalloc(*c, ctr.size() * 8);
      ck(cudaMemcpy(c->l_ctr, ctr.data(), ctr.size() * 8, cudaMemcpyHostToDevice), "copy centres");
    } else {
      c->l_no = c->pat.NO;
      c->l_ctr = nullptr;
      c->l_nbr = (int*)dalloc(*c, (size_t)ne * c->pat.NO * 4);
      ck(cudaMemcpy(c->l_nbr, c->host[0].nbr.data(), (size_t)ne * c->pat.NO * 4, cudaMemcpyHostToDevice),
         "copy nbr");
    }
    c->lF = (float*)dalloc(*c, (size_t)ne * c->l_ldf * 4);
    c->lH = (float*)dalloc(*c, (size_t)ne * hidden * 4);
    c->lY = (float*)dalloc(*c, (size_t)ne * nb * 4);
    c->lnrm = (float*)dalloc(*c, (size_t)ne * 4);
    c->lxt = (float*)dalloc(*c, (size_t)ne * nb * 4);
    c->lrt = (float*)dalloc(*c, (size_t)ne * nb * 4);
    c->lsums = (double*)dalloc(*c, 1024 * 8);
    c->lTg = (float*)dalloc(*c, (size_t)ne * nb * 4);
    c->l_acc = c->l_rej = 0;
    c->lF2 = (float*)dalloc(*c, (size_t)ne * hidden * 4);
    c->l_zero = (float*)dalloc(*c, (size_t)ne * nb * 4);
    ck(cudaMemset(c->l_zero, 0, (size_t)ne * nb * 4), "memset");
    c->lTX = c->lTT = c->lTE = nullptr;
    c->l_rows = c->l_cap = 0;
    invalidate_graphs(*c);
    return STK_OK;
  });
}

int stk_learn_generate(stk_ctx* c, int nseeds, int cycles, uint64_t seed) {
  return guard(c, [&]() -> int {
    if (!c->lW1) return fail(c, STK_ERR_NOT_SETUP, "call stk_learn_setup first");
    if (nseeds < 1 || cycles < 1) return fail(c, STK_ERR_INVALID_ARG, "bad sample counts");
    const int nb = c->nb, ne = c->dev[0].ne, prec = c->precision;
    DevLevel& D0 = c->dev[0];
    cudaStream_t st = c->stream;
    const int64_t nvec = (int64_t)ne * nb;
    int64_t need = (int64_t)nseeds * cycles;
    if (need > c->l_cap) {
      c->lTX = (float*)dalloc(*c, (size_t)need * nvec * 4);
      c->lTE = (float*)dalloc(*c, (size_t)need * nvec * 4);
      c->l_cap = need;
    }
    c->l_rows = 0;
    const int* ndev = c->l_ndev;
    float* xs = (float*)dalloc(*c, (size_t)nvec * 4);
    float* bb = (float*)dalloc(*c, (size_t)nvec * 4);
    float* zero = (float*)dalloc(*c, (size_t)nvec * 4);
    ck(cudaMemsetAsync(zero, 0, (size_t)nvec * 4, st), "memset");
    int on = c->learn_on;
    c->learn_on = 0;   // states come from the plain V-cycle
    for (int sd = 0; sd < nseeds; ++sd) {
      ck(launch_smooth_field(ne, nb, c->s, c->d, ndev, c->l_ctr, seed + 7919ULL * sd, xs, st), "field");
      // b = A x*: the residual of x* against a zero right-hand side is -A x*.
      ck(run_element(*c, 0, prec, MODE_RESID, 0, ne, D0.dia[prec], zero, xs, D0.vr[1], st), "matvec");
      ck(launch_scale_f(nvec, -1.f, (const float*)D0.vr[1], bb, st), "negate");
      float* x = (float*)D0.vx[1];
      ck(cudaMemsetAsync(x, 0, (size_t)nvec * 4, st), "memset");
      for (int k = 0; k < cycles; ++k) {
        enqueue_cycle(*c, prec, 0, x, bb, st);
        // the residual the correction would see after this cycle's post-smoothing
        ck(run_element(*c, 0, prec, MODE_RESID, 0, ne, D0.dia[prec], bb, x, c->lTX + (size_t)c->l_rows * nvec, st),
           "residual");
        // and the error e = x* - x the cycle left (the supervised target)
        float* e = c->lTE + (size_t)c->l_rows * nvec;
        ck(launch_scale_f(nvec, -1.f, x, e, st), "error");
        ck(launch_axpy(0, 0, nvec, e, xs, st), "error");
        c->launches += 3;
        c->l_rows += 1;
      }
    }
    ck(cudaStreamSynchronize(st), "sync");
    c->learn_on = on;
    return STK_OK;
  });
}

int stk_learn_field(stk_ctx* c, uint64_t seed, double* x, void* stream) {
  return guard(c, [&]() -> int {
    if (!c->lW1) return fail(c, STK_ERR_NOT_SETUP, "call stk_learn_setup first");
    if (!x) return fail(c, STK_ERR_INVALID_ARG, "null vector");
    cudaStream_t st = (cudaStream_t)stream;
    const int ne = c->dev[0].ne, nb = c->nb;
    float* xs = (float*)c->lxt;   // scratch of the learned smoother, [ne][nb]
    ck(launch_smooth_field(ne, nb, c->s, c->d, c->l_ndev, c->l_ctr, seed, xs, st), "field");
    ck(launch_convert(1, 0, (int64_t)ne * nb, x, xs, st), "convert");
    c->launches += 2;
    ck(cudaStreamSynchronize(st), "sync");
    return STK_OK;
  });
}

// Loss ||r - A delta||^2 / ||r||^2 of one residual state and its gradient
// (packed like the weights) in c.lgrad; the loss goes to *loss_dev (device).
// delta_i = ||r_i|| MLP(features_i); A is symmetric, so d loss / d delta =
// -2 A q / ||r||^2 with q = r - A delta, and A q is minus the residual of q
// against a zero right-hand side.
void enqueue_residual_loss_grad(Ctx& c, const float* r, double* sums, cudaStream_t st) {
  DevLevel& D0 = c.dev[0];
  const int ne = D0.ne, nb = c.nb, H = c.l_hid, IN = c.l_in, ldf = c.l_ldf, prec = c.precision;
  const int64_t nvec = (int64_t)ne * nb;
  float* gW1 = c.lgrad;
  float* gb1 = gW1 + (int64_t)IN * H;
  float* gW2 = gb1 + H;
  float* gb2 = gW2 + (int64_t)H * nb;
  ck(launch_features(ne, nb, 2 * c.d, c.l_no, ldf, c.l_nbr, r, c.lF, c.lnrm, st), "features");
  ck(launch_sgemm(ne, H, IN, 0, 0, c.lF, ldf, c.lW1, H, c.lH, H, c.lb1, 1, 1.f, 0.f, st), "fwd1");
  ck(launch_sgemm(ne, nb, H, 0, 0, c.lH, H, c.lW2, nb, c.lY, nb, c.lb2, 0, 1.f, 0.f, st), "fwd2");
  ck(cudaMemsetAsync(c.lrt, 0, (size_t)nvec * 4, st), "memset");
  ck(launch_apply_correction(ne, nb, nb, c.lrt, c.lnrm, c.lY, c.lxt, st), "delta");       // lxt = delta
  ck(run_element(c, 0, prec, MODE_RESID, 0, ne, D0.dia[prec], r, c.lxt, c.lrt, st), "q");  // lrt = q
  ck(launch_sumsq_f(nvec, r, sums + 16, sums, st), "||r||");
  ck(launch_sumsq_f(nvec, c.lrt, sums + 16, sums + 1, st), "||q||");
  // g = 2 (-A q) / ||r||^2 into lxt (reusing delta's buffer), then dY = ||r_i|| g_i.
  ck(run_element(c, 0, prec, MODE_RESID, 0, ne, D0.dia[prec], c.l_zero, c.lrt, c.lxt, st), "-A q");
  ck(launch_scale_by_norm(nvec, sums, c.lxt, st), "scale");
  ck(cudaMemsetAsync(c.lrt, 0, (size_t)nvec * 4, st), "memset");
  ck(launch_apply_correction(ne, nb, nb, c.lrt, c.lnrm, c.lxt, c.lY, st), "dY");          // lY = dY
  ck(launch_sgemm(H, nb, ne, 1, 0, c.lH, H, c.lY, nb, gW2, nb, nullptr, 0, 1.f, 0.f, st), "gW2");
  ck(launch_colsum(ne, nb, c.lY, nb, gb2, 1.f, st), "gb2");
  ck(launch_sgemm(ne, H, nb, 0, 1, c.lY, nb, c.lW2, nb, c.lF2, H, nullptr, 0, 1.f, 0.f, st), "dH");
  ck(launch_tanh_back((int64_t)ne * H, c.lH, c.lF2, st), "tanh'");
  ck(launch_sgemm(IN, H, ne, 1, 0, c.lF, ldf, c.lF2, H, gW1, H, nullptr, 0, 1.f, 0.f, st), "gW1");
  ck(launch_colsum(ne, H, c.lF2, H, gb1, 1.f, st), "gb1");
  c.launches += 18;
}

// Supervised objective on one stored state: features of r, y = MLP, target
// t_i = e_i / ||r_i||, loss = sum_i ||y_i - t_i||^2 / ne (sums[1] / sums[0]
// with sums[0] = ne), and its gradient (packed like the weights) in c.lgrad.
void enqueue_supervised_loss_grad(Ctx& c, const float* r, const float* e, double* sums, cudaStream_t st) {
  DevLevel& D0 = c.dev[0];
  const int ne = D0.ne, nb = c.nb, H = c.l_hid, IN = c.l_in, ldf = c.l_ldf;
  const int64_t nvec = (int64_t)ne * nb;
  float* gW1 = c.lgrad;
  float* gb1 = gW1 + (int64_t)IN * H;
  float* gW2 = gb1 + H;
  float* gb2 = gW2 + (int64_t)H * nb;
  ck(launch_features(ne, nb, 2 * c.d, c.l_no, ldf, c.l_nbr, r, c.lF, c.lnrm, st), "features");
  ck(launch_sgemm(ne, H, IN, 0, 0, c.lF, ldf, c.lW1, H, c.lH, H, c.lb1, 1, 1.f, 0.f, st), "fwd1");
  ck(launch_sgemm(ne, nb, H, 0, 0, c.lH, H, c.lW2, nb, c.lY, nb, c.lb2, 0, 1.f, 0.f, st), "fwd2");
  ck(launch_target(ne, nb, nb, e, c.l_zero, c.lnrm, c.lTg, st), "targets");
  ck(launch_mse_grad(nvec, 1.f / (float)ne, c.lY, c.lTg, c.lY, sums + 16, sums + 1, st), "mse");   // lY = dY
  ck(launch_fill(sums, (double)ne, st), "rows");
  ck(launch_sgemm(H, nb, ne, 1, 0, c.lH, H, c.lY, nb, gW2, nb, nullptr, 0, 1.f, 0.f, st), "gW2");
  ck(launch_colsum(ne, nb, c.lY, nb, gb2, 1.f, st), "gb2");
  ck(launch_sgemm(ne, H, nb, 0, 1, c.lY, nb, c.lW2, nb, c.lF2, H, nullptr, 0, 1.f, 0.f, st), "dH");
  ck(launch_tanh_back((int64_t)ne * H, c.lH, c.lF2, st), "tanh'");
  ck(launch_sgemm(IN, H, ne, 1, 0, c.lF, ldf, c.lF2, H, gW1, H, nullptr, 0, 1.f, 0.f, st), "gW1");
  ck(launch_colsum(ne, H, c.lF2, H, gb1, 1.f, st), "gb1");
  c.launches += 13;
}

void enqueue_loss_grad(Ctx& c, int64_t state, cudaStream_t st) {
  const int64_t nvec = (int64_t)c.dev[0].ne * c.nb;
  if (c.l_objective == 1)
    enqueue_supervised_loss_grad(c, c.lTX + (size_t)state * nvec, c.lTE + (size_t)state * nvec, c.lsums, st);
  else
    enqueue_residual_loss_grad(c, c.lTX + (size_t)state * nvec, c.lsums, st);
}

int stk_learn_train(stk_ctx* c, int epochs, int batch, double lr, uint64_t seed, double* loss_out) {
  return guard(c, [&]() -> int {
    if (!c->lW1) return fail(c, STK_ERR_NOT_SETUP, "call stk_learn_setup first");
    if (c->l_rows <= 0) return fail(c, STK_ERR_NOT_SETUP, "call stk_learn_generate first");
    if (epochs < 1 || !(lr > 0)) return fail(c, STK_ERR_INVALID_ARG, "bad training options");
    (void)batch;
    cudaStream_t st = c->stream;
    const int64_t nvec = (int64_t)c->dev[0].ne * c->nb;
    uint64_t z = seed;
    double sum_loss = 0.0;
    int nloss = 0;
    for (int ep = 0; ep < epochs; ++ep) {
      sum_loss = 0.0;
      nloss = 0;
      for (int64_t k = 0; k < c->l_rows; ++k) {
        z = z * 6364136223846793005ULL + 1442695040888963407ULL;
        const int64_t state = (int64_t)((z >> 33) % (uint64_t)c->l_rows);
        enqueue_loss_grad(*c, state, st);
        c->l_adam_t++;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, (float)c->l_adam_t), c2 = 1.f - std::pow(b2, (float)c->l_adam_t);
        ck(launch_adam(c->l_nparam, (float)lr, b1, b2, c1, c2, 1e-8f, c->lW1, c->lgrad, c->lm, c->lv, st), "adam");
        c->launches++;
        double h[2];
        ck(cudaMemcpyAsync(h, c->lsums, 2 * sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
        ck(cudaStreamSynchronize(st), "sync");
        sum_loss += h[1] / h[0];
        ++nloss;
      }
    }
    if (loss_out) *loss_out = nloss ? sum_loss / nloss : 0.0;
    return STK_OK;
  });
}

int stk_learn_infer(stk_ctx* c, const float* r, float* y, float* nrm) {
  return guard(c, [&]() -> int {
    if (!c->lW1) return fail(c, STK_ERR_NOT_SETUP, "call stk_learn_setup first");
    if (!r || !y || !nrm) return fail(c, STK_ERR_INVALID_ARG, "null vector");
    const int ne = c->dev[0].ne, nb = c->nb;
    cudaStream_t st = c->stream;
    ck(launch_features(ne, nb, 2 * c->d, c->l_no, c->l_ldf, c->l_nbr, r, c->lF, nrm, st), "features");
    ck(launch_sgemm(ne, c->l_hid, c->l_in, 0, 0, c->lF, c->l_ldf, c->lW1, c->l_hid, c->lH, c->l_hid, c->lb1, 1, 1.f,
                    0.f, st),
       "layer 1");
    ck(launch_sgemm(ne, nb, c->l_hid, 0, 0, c->lH, c->l_hid, c->lW2, nb, y, nb, c->lb2, 0, 1.f, 0.f, st), "layer 2");
    c->launches += 3;
    ck(cudaStreamSynchronize(st), "sync");
    return STK_OK;
  });
}

int stk_learn_state(stk_ctx* c, int64_t state, float* r) {
  return guard(c, [&]() -> int {
    if (!c->lTX || state < 0 || state >= c->l_rows || !r) return fail(c, STK_ERR_INVALID_ARG, "bad state index");
    const int64_t nvec = (int64_t)c->dev[0].ne * c->nb;
    ck(cudaMemcpy(r, c->lTX + (size_t)state * nvec, (size_t)nvec * 4, cudaMemcpyDeviceToHost), "copy");
    return STK_OK;
  });
}

int stk_learn_error_state(stk_ctx* c, int64_t state, float* e) {
  return guard(c, [&]() -> int {
    if (!c->lTE || state < 0 || state >= c->l_rows || !e) return fail(c, STK_ERR_INVALID_ARG, "bad state index");
    const int64_t nvec = (int64_t)c->dev[0].ne * c->nb;
    ck(cudaMemcpy(e, c->lTE + (size_t)state * nvec, (size_t)nvec * 4, cudaMemcpyDeviceToHost), "copy");
    return STK_OK;
  });
}

int stk_learn_objective(stk_ctx* c, int objective) {
  return guard(c, [&]() -> int {
    if (objective != 0 && objective != 1) return fail(c, STK_ERR_INVALID_ARG, "objective must be 0 or 1");
    c->l_objective = objective;
    return STK_OK;
  });
}

int stk_learn_history(stk_ctx* c, int* decision, double* ratio, int max, int* count, double* kappa_out) {
  return guard(c, [&]() -> int {
    const int n = (int)c->l_hist.size();
    for (int k = 0; k < n && k < max; ++k) {
      if (decision) decision[k] = c->l_hist[k];
      if (ratio) ratio[k] = c->l_ratio[k];
    }
    if (count) *count = n;
    if (kappa_out) *kappa_out = c->l_kappa;
    return STK_OK;
  });
}

int stk_learn_grad(stk_ctx* c, int64_t state, float* grad, double* loss_out) {
  return guard(c, [&]() -> int {
    if (!c->lTX || state < 0 || state >= c->l_rows || !grad) return fail(c, STK_ERR_INVALID_ARG, "bad state index");
    cudaStream_t st = c->stream;
    enqueue_loss_grad(*c, state, st);
    double h[2];
    ck(cudaMemcpyAsync(h, c->lsums, 2 * sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaMemcpyAsync(grad, c->lgrad, c->l_nparam * 4, cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaStreamSynchronize(st), "sync");
    if (loss_out) *loss_out = h[1] / h[0];
    return STK_OK;
  });
}

int stk_learn_enable(stk_ctx* c, int on) {
  return guard(c, [&]() -> int {
    if (on && !c->lW1) return fail(c, STK_ERR_NOT_SETUP, "call stk_learn_setup first");
    c->learn_on = on ? 1 : 0;
    invalidate_graphs(*c);
    c->l_acc = c->l_rej = 0;
    return STK_OK;
  });
}

int stk_learn_sizes(stk_ctx* c, int* in, int* hidden, int* out, int64_t* nparam, int64_t* rows) {
  return guard(c, [&]() -> int {
    if (!c->lW1) return fail(c, STK_ERR_NOT_SETUP, "call stk_learn_setup first");
    if (in) *in = c->l_in;
    if (hidden) *hidden = c->l_hid;
    if (out) *out = c->nb;
    if (nparam) *nparam = c->l_nparam;
    if (rows) *rows = c->l_rows;
    return STK_OK;
  });
}

int stk_learn_stats(stk_ctx* c, int64_t* accepted, int64_t* rejected) {
  return guard(c, [&]() -> int {
    if (accepted) *accepted = c->l_acc;
    if (rejected) *rejected = c->l_rej;
    return STK_OK;
  });
}

int stk_learn_weights(stk_ctx* c, float* host, int64_t count, int direction) {
  return guard(c, [&]() -> int {
    if (!c->lW1) return fail(c, STK_ERR_NOT_SETUP, "call stk_learn_setup first");
    if (!host || count != c->l_nparam) return fail(c, STK_ERR_INVALID_ARG, "weight count mismatch");
    if (direction == 0)
      ck(cudaMemcpy(host, c->lW1, count * 4, cudaMemcpyDeviceToHost), "copy weights");
    else {
      ck(cudaMemcpy(c->lW1, host, count * 4, cudaMemcpyHostToDevice), "copy weights");
      invalidate_graphs(*c);
    }
    return STK_OK;
  });
}

int stk_set_levelset_circle(stk_ctx* c, double cx, double cy, double r) {
  return guard(c, [&]() -> int {
    if (c->d != 2) return fail(c, STK_ERR_INVALID_ARG, "set a 2D mesh first");
    if (!std::isfinite(cx) || !std::isfinite(cy) || !std::isfinite(r) || r < 0)
      return fail(c, STK_ERR_INVALID_ARG, "bad circle");
    free_device(*c);
    c->cutg.reset();
    c->cuts.reset();
    if (r == 0) {
      c->cut = 0;
      c->cut_inside = 0;
      c->mu_phase.clear();
      c->rho_phase.clear();
      c->cut_delta = 0.0;
      return STK_OK;
    }
    c->cut = 1;
    c->cut_c[0] = cx;
    c->cut_c[1] = cy;
    c->cut_r = r;
    c->chi.clear();
    return STK_OK;
  });
}

int stk_set_element_warps(stk_ctx* c, int warps) {
  return guard(c, [&]() -> int {
    if (warps != 0 && warps != 1 && warps != 2 && warps != 4)
      return fail(c, STK_ERR_INVALID_ARG, "warps per element: 0 (by launch size), 1, 2 or 4");
    c->gen_warps = warps;
    invalidate_graphs(*c);
    return STK_OK;
  });
}

int stk_set_phase_density(stk_ctx* c, const double* rho_phase, double delta) {
  return guard(c, [&]() -> int {
    if (!c->cut) return fail(c, STK_ERR_INVALID_ARG, "phase densities belong to cut-cell meshes");
    if (!(delta >= 0) || !std::isfinite(delta)) return fail(c, STK_ERR_INVALID_ARG, "delta must be >= 0");
    free_device(*c);
    if (delta == 0) {
      c->rho_phase.clear();
      c->cut_delta = 0.0;
      return STK_OK;
    }
    if (!rho_phase) return fail(c, STK_ERR_INVALID_ARG, "null densities");
    const int np = c->cut_inside ? 1 : 2;   // one per phase of stk_set_phases
    for (int i = 0; i < np; ++i)
      if (!(rho_phase[i] > 0) || !std::isfinite(rho_phase[i]))
        return fail(c, STK_ERR_INVALID_ARG, "phase density must be finite and positive");
    c->rho_phase.assign(rho_phase, rho_phase + np);
    c->cut_delta = delta;
    return STK_OK;
  });
}

int stk_set_phases(stk_ctx* c, int nphase, const int* chi, const double* mu_phase, int scale) {
  return guard(c, [&]() -> int {
    if (c->p < 0) return fail(c, STK_ERR_INVALID_ARG, "set mesh and discretisation first");
    free_device(*c);
    if (nphase == 0) {
      c->chi.clear();
      c->mu_phase.clear();
      c->scale_mu = 0;
      return STK_OK;
    }
    if (c->cut) {
      // embedded circle: phase 1 inside, 2 outside (nphase = 2), or the disc
      // alone with Dirichlet data on the circle (nphase = 1); no element phase array
      if ((nphase != 1 && nphase != 2) || !mu_phase)
        return fail(c, STK_ERR_INVALID_ARG, "the embedded circle takes two phases, or one (the disc alone)");
      for (int i = 0; i < nphase; ++i)
        if (!(mu_phase[i] > 0) || !std::isfinite(mu_phase[i]))
          return fail(c, STK_ERR_INVALID_ARG, "phase viscosity must be finite and positive");
      c->chi.clear();
      c->mu_phase.assign(mu_phase, mu_phase + nphase);
      c->cut_inside = nphase == 1 ? 1 : 0;
      c->rho_phase.clear();
      c->cut_delta = 0.0;
      c->cutg.reset();
      c->cuts.reset();
      c->scale_mu = scale ? 1 : 0;
      return STK_OK;
    }
    if (nphase < 1 || nphase > 64 || !chi || !mu_phase) return fail(c, STK_ERR_INVALID_ARG, "bad phase arguments");
    int64_t ne = 1;
    for (int k = 0; k < c->d; ++k) ne *= c->n[k];
    for (int64_t e = 0; e < ne; ++e)
      if (chi[e] < 1 || chi[e] > nphase) return fail(c, STK_ERR_INVALID_ARG, "phase index out of range");
    for (int i = 0; i < nphase; ++i)
      if (!(mu_phase[i] > 0) || !std::isfinite(mu_phase[i]))
        return fail(c, STK_ERR_INVALID_ARG, "phase viscosity must be finite and positive");
    c->chi.assign(chi, chi + ne);
    c->mu_phase.assign(mu_phase, mu_phase + nphase);
    c->scale_mu = scale ? 1 : 0;
    return STK_OK;
  });
}

int stk_get_interface(stk_ctx* c, int* chi_minus, int* chi_plus, double* normals) {
  return guard(c, [&]() -> int {
    if (c->p < 0) return fail(c, STK_ERR_INVALID_ARG, "set mesh and discretisation first");
    if (c->cut) return fail(c, STK_ERR_INVALID_ARG, "cut-cell meshes: interface points are kind STK_PTS_INTERFACE");
    std::vector<int> cm, cp;
    std::vector<double> nr;
    interface_info(*c, cm, cp, nr);
    if (chi_minus) std::copy(cm.begin(), cm.end(), chi_minus);
    if (chi_plus) std::copy(cp.begin(), cp.end(), chi_plus);
    if (normals) std::copy(nr.begin(), nr.end(), normals);
    return STK_OK;
  });
}

int stk_assemble_rhs2(stk_ctx* c, const double* f_vol, const double* bdata, const double* idata, double* b) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (!f_vol || !b) return fail(c, STK_ERR_INVALID_ARG, "null argument");
    if (c->cut) {
      if (!bdata || !idata) return fail(c, STK_ERR_INVALID_ARG, "null boundary or interface data");
      std::string err;
      const int rc = cut_assemble_rhs(*c, f_vol, bdata, idata, b, err);
      return rc == STK_OK ? rc : fail(c, rc, err);
    }
    if (count_points(*c, 2) > 0 && !bdata) return fail(c, STK_ERR_INVALID_ARG, "null boundary data");
    return assemble_rhs_host2(*c, f_vol, bdata, idata, b);
  });
}

int stk_get_colours(stk_ctx* c, int level, int* colours) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (level < 0 || level >= nlevels(*c) - 1 || !colours) return fail(c, STK_ERR_INVALID_ARG, "bad level");
    const DevLevel& D = c->dev[level];
    std::vector<int> perm(D.ne);
    ck(cudaMemcpy(perm.data(), D.perm, D.ne * sizeof(int), cudaMemcpyDeviceToHost), "copy perm");
    for (int col = 0; col < D.ncolour; ++col)
      for (int pos = D.cstart[col]; pos < D.cstart[col + 1]; ++pos) colours[perm[pos]] = col;
    return STK_OK;
  });
}

int stk_get_scaling(stk_ctx* c, double* D) {
  return guard(c, [&]() -> int {
    if (!c->ready) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    if (!D) return fail(c, STK_ERR_INVALID_ARG, "null argument");
    const HostLevel& H = c->host[0];
    if (H.Dscale.empty())
      std::fill(D, D + (size_t)H.ne * c->nb, 1.0);
    else
      std::copy(H.Dscale.begin(), H.Dscale.end(), D);
    return STK_OK;
  });
}

int stk_fp64_fma_rate(stk_ctx* c, double* tflops, void* stream) {
  return guard(c, [&]() -> int {
    if (!tflops) return fail(c, STK_ERR_INVALID_ARG, "null output");
    ck(cudaSetDevice(c->device), "cudaSetDevice");
    int sms = 0;
    ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device), "attribute");
    const int blocks = sms * 8, iters = 1 << 16;
    if (!c->norm_buf) return fail(c, STK_ERR_NOT_SETUP, "call stk_setup first");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    ck(cudaEventCreate(&e0), "event");
    ck(cudaEventCreate(&e1), "event");
    double best = 0.0;
    for (int rep = 0; rep < 4; ++rep) {
      ck(cudaEventRecord(e0, st), "record");
      ck(launch_fp64_fma(blocks, iters, c->norm_buf + 1048, st), "fp64 probe");
      ck(cudaEventRecord(e1, st), "record");
      ck(cudaEventSynchronize(e1), "sync");
      float ms = 0.f;
      ck(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
      const double flops = 2.0 * 8.0 * iters * (double)blocks * 256.0;
      if (rep > 0 && ms > 0) best = std::max(best, flops / (ms * 1e-3) / 1e12);   // rep 0 warms up
      c->launches++;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *tflops = best;
    return STK_OK;
  });
}

int stk_launch_count(stk_ctx* c, int64_t* count) {
  if (!c || !count) return STK_ERR_INVALID_ARG;
  *count = c->launches;
  return STK_OK;
}

int stk_solve_batch_persistent(stk_ctx* const* ctx, int n, double* const* x, const double* const* b, double rtol,
                               int maxit, int ctas_per_sm, int* iters_out, int* status_out, double* hist,
                               void* stream) {
  if (!ctx || !x || !b || n < 1 || n > 4096 || maxit < 0 || !(rtol > 0) || ctas_per_sm < 1 || ctas_per_sm > 8)
    return STK_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    if (!ctx[i] || !x[i] || !b[i]) return STK_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (ctx[j] == ctx[i]) return STK_ERR_INVALID_ARG;
  }
  stk_ctx* c0 = ctx[0];
  return guard(c0, [&]() -> int {
    for (int i = 0; i < n; ++i) {
      Ctx& c = *ctx[i];
      if (!c.ready) return fail(c0, STK_ERR_NOT_SETUP, "problem " + std::to_string(i) + " is not set up");
      if (c.device != c0->device) return fail(c0, STK_ERR_INVALID_ARG, "problems on different devices");
      if (c.cut) return fail(c0, STK_ERR_INVALID_ARG, "the persistent batch takes Cartesian problems");
      if (c.precision != STK_FP32)
        return fail(c0, STK_ERR_INVALID_ARG, "the persistent batch runs FP32-record cycles (problem " +
                                                 std::to_string(i) + ")");
      if (c.cluster_on)
        return fail(c0, STK_ERR_INVALID_ARG, "the persistent batch smooths element by element (problem " +
                                                 std::to_string(i) + " clusters its finest level)");
      const int sv = c.pat.s;
      if (sv != 4 && sv != 8 && sv != 9 && sv != 16 && sv != 27)
        return fail(c0, STK_ERR_INVALID_ARG, "degree not compiled into the persistent batch");
    }
    ck(cudaSetDevice(c0->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    ck(cudaStreamSynchronize(st), "sync caller stream");
    // ||b|| and the initial residual of every problem (its own stream)
    std::vector<double> bnorm(n), rel0(n);
    for (int i = 0; i < n; ++i) {
      Ctx& c = *ctx[i];
      enqueue_norm(c, b[i], c.stream);
      ck(cudaStreamSynchronize(c.stream), "sync");
      bnorm[i] = std::sqrt(c.norm_host[0]);
      if (bnorm[i] == 0.0) bnorm[i] = 1.0;
      enqueue_residual64(c, x[i], b[i], c.r64, c.stream);
      enqueue_norm(c, c.r64, c.stream);
      ck(cudaStreamSynchronize(c.stream), "sync");
      rel0[i] = std::sqrt(c.norm_host[0]) / bnorm[i];
    }
    // per-problem programs: cycle input, V-cycle, x += c, FP64 residual, norm, check
    std::vector<std::vector<CyclePhase>> progs(n);
    int64_t nchunk_total = 0;
    std::vector<int64_t> part_off(n);
    for (int i = 0; i < n; ++i) {
      Ctx& c = *ctx[i];
      DevLevel& D0 = c.dev[0];
      const int64_t n0 = level_ne(c, 0) * c.nb, nch = (n0 + kBatchChunk - 1) / kBatchChunk;
      part_off[i] = nchunk_total;
      nchunk_total += nch;
      std::vector<CyclePhase>& pr = progs[i];
      CyclePhase cv{};
      cv.op = PHASE_CONVERT;
      cv.n = nch;
      cv.in = c.r64;
      cv.out = D0.vb[1];
      cv.xz = D0.vx[1];
      pr.push_back(cv);
      emit_cycle_phases(c, STK_FP32, 0, pr);
      CyclePhase ax{};
      ax.op = PHASE_AXPY;
      ax.n = nch;
      ax.in = D0.vx[1];
      ax.out = x[i];
      pr.push_back(ax);
      CyclePhase rr{};
      rr.op = PHASE_RESID64;
      rr.n = D0.ne;
      rr.cpl = D0.cpl[0];
      rr.mat = D0.dia[0];
      rr.perm = D0.perm;
      rr.nbr = D0.nbr;
      rr.b = b[i];
      rr.x = x[i];
      rr.r = c.r64;
      pr.push_back(rr);
      CyclePhase nm{};
      nm.op = PHASE_NORM;
      nm.n = nch;
      nm.in = c.r64;
      pr.push_back(nm);
      CyclePhase ch{};
      ch.op = PHASE_CHECK;
      ch.n = 1;
      pr.push_back(ch);
    }
    // steps: phase k of every problem that has one, run together
    size_t nsteps = 0;
    for (auto& pr : progs) nsteps = std::max(nsteps, pr.size());
    std::vector<BatchStep> steps(nsteps);
    std::vector<BatchTask> tasks;
    auto units_of = [](const CyclePhase& ph) -> int64_t {
      return ph.n;   // every unit is one warp's: element, coarse element, bottom row or vector chunk
    };
    for (size_t k = 0; k < nsteps; ++k) {
      steps[k].t0 = (int)tasks.size();
      int64_t u = 0;
      for (int i = 0; i < n; ++i) {
        if (k >= progs[i].size()) continue;
        BatchTask t{};
        t.prob = i;
        t.ustart = u;
        t.ph = progs[i][k];
        u += units_of(t.ph);
        tasks.push_back(t);
      }
      steps[k].t1 = (int)tasks.size();
      steps[k].units = u;
    }
    // device copies: problems, steps, tasks, partials, flags, histories
    struct DevBuf {
      std::vector<void*> p;
      ~DevBuf() {
        for (void* q : p) cudaFree(q);
      }
      void* get(size_t bytes) {
        void* q = nullptr;
        if (cudaMalloc(&q, bytes ? bytes : 16) != cudaSuccess) throw CudaFail{cudaErrorMemoryAllocation, "cudaMalloc"};
        p.push_back(q);
        return q;
      }
    } buf;
    double* part = (double*)buf.get((size_t)nchunk_total * 8);
    int* flags = (int*)buf.get((size_t)3 * n * sizeof(int));   // active, iters, status
    double* dhist = (double*)buf.get((size_t)n * (maxit + 1) * 8);
    std::vector<int> hflags(3 * n, 0);
    std::vector<double> hh((size_t)n * (maxit + 1), 0.0);
    std::vector<BatchProblem> probs(n);
    size_t smem = 0;
    for (int i = 0; i < n; ++i) {
      Ctx& c = *ctx[i];
      BatchProblem& B = probs[i];
      B.pat = c.pat;
      B.n0 = level_ne(c, 0) * c.nb;
      B.x64 = x[i];
      B.r64 = c.r64;
      B.part = part + part_off[i];
      B.bnorm = bnorm[i];
      B.rel0 = rel0[i];
      B.active = flags + i;
      B.iters = flags + n + i;
      B.status = flags + 2 * n + i;
      B.hist = dhist + (size_t)i * (maxit + 1);
      hflags[i] = (rel0[i] > rtol && maxit > 0) ? 1 : 0;
      hh[(size_t)i * (maxit + 1)] = rel0[i];
      smem = std::max(smem, batch_smem_bytes(c.pat));
    }
    BatchProblem* dprobs = (BatchProblem*)buf.get(probs.size() * sizeof(BatchProblem));
    BatchStep* dsteps = (BatchStep*)buf.get(steps.size() * sizeof(BatchStep));
    BatchTask* dtasks = (BatchTask*)buf.get(tasks.size() * sizeof(BatchTask));
    ck(cudaMemcpy(dprobs, probs.data(), probs.size() * sizeof(BatchProblem), cudaMemcpyHostToDevice), "copy");
    ck(cudaMemcpy(dsteps, steps.data(), steps.size() * sizeof(BatchStep), cudaMemcpyHostToDevice), "copy");
    ck(cudaMemcpy(dtasks, tasks.data(), tasks.size() * sizeof(BatchTask), cudaMemcpyHostToDevice), "copy");
    ck(cudaMemcpy(flags, hflags.data(), hflags.size() * sizeof(int), cudaMemcpyHostToDevice), "copy");
    ck(cudaMemcpy(dhist, hh.data(), hh.size() * 8, cudaMemcpyHostToDevice), "copy");
    ck(cudaMemsetAsync(c0->gbar, 0, sizeof(GridBarrierWords), st), "memset");
    ck(cudaMemsetAsync(c0->dev_err, 0, sizeof(int), st), "memset");
    int sms = 0;
    ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c0->device), "attribute");
    ck(launch_batch_solve(dprobs, n, dsteps, (int)nsteps, dtasks, maxit, rtol, 0, smem, c0->gbar, c0->dev_err,
                          c0->barrier_limit, sms * ctas_per_sm, st),
       "persistent batch launch");
    c0->launches++;
    int err = 0;
    ck(cudaMemcpyAsync(&err, c0->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaStreamSynchronize(st), "sync");
    ck(cudaMemcpy(hflags.data(), flags, hflags.size() * sizeof(int), cudaMemcpyDeviceToHost), "copy");
    ck(cudaMemcpy(hh.data(), dhist, hh.size() * 8, cudaMemcpyDeviceToHost), "copy");
    if (err != 0) {
      ck(cudaMemset(c0->dev_err, 0, sizeof(int)), "memset");
      return fail(c0, STK_ERR_TIMEOUT, "a grid-barrier wait of the persistent batch reached its bound");
    }
    int rc = STK_OK;
    for (int i = 0; i < n; ++i) {
      const int it = hflags[n + i];
      const int stt = hflags[2 * n + i];
      if (iters_out) iters_out[i] = it;
      if (status_out) status_out[i] = stt;
      if (hist)
        for (int k = 0; k <= maxit; ++k) hist[(size_t)i * (maxit + 1) + k] = k <= it ? hh[(size_t)i * (maxit + 1) + k] : 0.0;
      if (rc == STK_OK && stt != STK_OK) rc = stt;
    }
    if (rc != STK_OK) return fail(c0, rc, "a problem of the batch diverged");
    return STK_OK;
  });
}

int stk_solve_batch(stk_ctx* const* ctx, int n, double* const* x, const double* const* b, int nrhs, double rtol,
                    int maxit, int inner, int threads, int* iters_out, int* status_out, void* stream) {
  if (!ctx || !x || !b || n < 1 || nrhs < 1 || nrhs > 8) return STK_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    if (!ctx[i] || !x[i] || !b[i]) return STK_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (ctx[j] == ctx[i]) return STK_ERR_INVALID_ARG;   // one context serves one problem at a time
  }
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return STK_ERR_CUDA;
  int nt = threads > 0 ? threads : (int)std::max(1u, std::thread::hardware_concurrency());
  nt = std::min(nt, n);
  std::vector<int> status(n, STK_OK), iters(n, 0);
  std::atomic<int> next(0);
  // Each worker takes the next unsolved problem and runs its whole outer
  // iteration on the problem's own context stream; the problems' kernels
  // therefore overlap on the GPU wherever one problem alone leaves it idle.
  auto worker = [&]() {
    for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1)) {
      if (cudaSetDevice(ctx[i]->device) != cudaSuccess) {
        status[i] = STK_ERR_CUDA;
        continue;
      }
      int it = 0;
      status[i] = nrhs == 1 ? stk_solve(ctx[i], x[i], b[i], rtol, maxit, &it, nullptr, nullptr)
                            : stk_solve_multi(ctx[i], x[i], b[i], nrhs, rtol, maxit, inner, &it, nullptr, nullptr);
      iters[i] = it;
    }
  };
  std::vector<std::thread> pool;
  try {
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  } catch (...) {
    // fewer workers than asked for: the ones started (and this thread) do the rest
  }
  worker();
  for (auto& th : pool) th.join();
  int rc = STK_OK;
  for (int i = 0; i < n; ++i) {
    if (iters_out) iters_out[i] = iters[i];
    if (status_out) status_out[i] = status[i];
    if (rc == STK_OK && status[i] != STK_OK) rc = status[i];
  }
  return rc;
}

}  // extern "C"
