// Internal data structures of the Stokes multigrid library (not part of the C ABI).
#pragma once

#include <atomic>
#include <functional>
#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace stk {

constexpr int kMaxTasks = 112;
constexpr int kMaxGather = 112;
constexpr int kMaxOffsets = 48;

// Coupling pattern of one element with its neighbours (identical on every
// level for given d and gamma).  A "task" is one s x s sub-block of the
// operator: row variable rv, column variable cv, neighbour offset slot.
struct Pattern {
  int d, s, nb;
  int T;       // number of coupling tasks (offset != 0)
  int TR;      // T * s task-rows
  int TRP;     // TR padded to a multiple of 8
  int NBP;     // nb padded to a multiple of 8
  int NO;      // number of distinct neighbour offsets
  int NG;      // number of distinct (offset, column variable) gathers
  int task_rv[kMaxTasks], task_cv[kMaxTasks], task_o[kMaxTasks], task_g[kMaxTasks];
  int rv_t0[5], rv_t1[5];           // tasks of row variable rv: [rv_t0, rv_t1)
  int g_o[kMaxGather], g_cv[kMaxGather];
  int off[kMaxOffsets][3];          // offset vectors
};

// One phase of the persistent coarse cycle (persist.cu): a data-parallel step
// of Algorithm 1 over n units, followed by a grid barrier.
enum PhaseOp {
  PHASE_GS = 0, PHASE_RESID = 1, PHASE_RESTRICT = 2, PHASE_PROLONG = 3, PHASE_BOTTOM = 4,
  // batched outer iteration (stk_solve_batch_persistent): FP64 residual on the
  // FP64 records, cycle input vb = (float) r64 with vx = 0, x64 += vx, partial
  // sums of ||r64||^2, and the per-problem convergence check
  PHASE_RESID64 = 5, PHASE_CONVERT = 6, PHASE_AXPY = 7, PHASE_NORM = 8, PHASE_CHECK = 9
};
struct CyclePhase {
  int op;
  int pos0;            // GS / RESID: first element position
  int64_t n;           // units: element positions, coarse elements, or bottom rows
  int dims[4];         // RESTRICT: nc0 nc1 nf0 nf1; PROLONG: nf0 nf1 nc0 nc1
  const void* cpl;     // GS / RESID records
  const void* mat;
  const int* perm;
  const int* nbr;
  const float* tsc;    // FP16 record scales
  const float* rsc;
  const void* b;
  void* x;
  void* r;
  const void* tr;      // RESTRICT: P, PROLONG: P^T, BOTTOM: pseudo-inverse
  const void* in;
  void* out;
  void* xz;            // RESTRICT: coarse iterate, zeroed in the same phase
};
// One problem of a persistent batch (device copy): its coupling pattern and
// shared-memory geometries, and the vectors of its outer iteration.
constexpr int kBatchChunk = 2048;   // entries per unit of the batch's vector phases
struct BatchProblem {
  Pattern pat;
  int64_t n0;           // level-0 unknowns
  double* x64;          // caller's iterate (FP64)
  double* r64;          // outer residual (context work vector)
  double* part;         // partial sums of ||r64||^2, one per chunk
  double bnorm, rel0;   // ||b|| and the initial relative residual
  int* active;          // 1 while iterating
  int* iters;           // outer iterations done
  int* status;          // 0, or STK_ERR_DIVERGED
  double* hist;         // relative residual after each iteration [maxit + 1]
};
// One step of a batch program: tasks [t0, t1) of the task table, run
// together; task t owns units [ustart[t], ustart[t + 1]) of the step.
struct BatchStep {
  int t0, t1;
  int64_t units;
};
struct BatchTask {
  int prob;
  int64_t ustart;
  CyclePhase ph;
};

// Grid barrier words (device): arrivals at the current barrier, barriers passed.
struct GridBarrierWords {
  unsigned int count;
  unsigned int gen;
};
constexpr int kErrBarrierTimeout = 2;   // error word value of an expired grid-barrier wait

// Host-side operators of one level, stored per element with offset slots.
//   slot 0: the element itself; slot 1+2k: offset -e_k; slot 2+2k: offset +e_k.
struct HostLevel {
  int n[3] = {1, 1, 1};
  int ne = 0;
  double h[3] = {0, 0, 0};
  double vol = 0;
  std::vector<double> M, Mmu, Mrho;     // [ne][s*s]
  std::vector<double> G;                // [d][ne][3][s*s]: G_k(e,e), G_k(e,e-e_k), G_k(e,e+e_k)
  std::vector<int> chi;                 // phase of every element (multi-phase problems)
  std::vector<double> Dscale;           // [ne][nb] sqrt(mu) diagonal scaling (when enabled)
  std::vector<double> Et, E, Emu, Erho; // [ne][1+2d][s*s]
  // Stokes operator blocks
  std::vector<double> D;                // [ne][nb*nb] diagonal blocks (row-major)
  std::vector<double> C;                // [ne][T][s*s] coupling task blocks (row-major)
  std::vector<int> nbr;                 // [ne][NO] neighbour element (-1 absent)
  // General block-sparse levels (cut-cell meshes): the coupling tasks of
  // element e are [tptr[e], tptr[e+1]), task t the s x s sub-block C[t] (rows
  // of variable tvar[t] / 4 of e, columns of variable tvar[t] % 4 of tnbr[t]);
  // the smoother colour of every element; and the injection to the next
  // coarser level (fine element e = Ib[e] times its parent's coefficients,
  // per variable).
  std::vector<int> tptr, tnbr, tvar;
  std::vector<int> colour;
  std::vector<int> parent;
  std::vector<double> Ib;               // [ne][s*s] row-major
};

// Device data of one level.
struct DevLevel {
  int ne = 0;
  int cstart[65] = {0};                 // colour ranges in colour-major positions
  int ncolour = 0;
  int* perm = nullptr;                  // [ne] position -> element
  int* nbr = nullptr;                   // [ne][NO] per position
  // per storage precision (FP64, FP32, BF16, FP16):
  void* cpl[4] = {nullptr, nullptr, nullptr, nullptr};   // [pos][s][TRP]
  void* inv[4] = {nullptr, nullptr, nullptr, nullptr};   // [pos][nb][NBP] column-major A_ii^{-1}
  void* dia[4] = {nullptr, nullptr, nullptr, nullptr};   // [pos][nb][NBP] column-major A_ii
  // power-of-two scales of the FP16 records: per coupling task [pos][T padded to 4],
  // per row of inv and of dia [pos][NBP]
  float* csc = nullptr;
  float* isc = nullptr;
  float* dsc = nullptr;
  // level 0 of a low-precision cycle: FP32 remainders of the FP64 coupling and
  // diagonal records (cpl[1] + cpl_lo, dia[1] + dia_lo carry ~48 bits)
  void* cpl_lo = nullptr;
  void* dia_lo = nullptr;
  // cycle vectors: index 0 FP64, index 1 FP32
  void* vx[2] = {nullptr, nullptr};
  void* vb[2] = {nullptr, nullptr};
  void* vr[2] = {nullptr, nullptr};
  // the same for several right-hand sides, interleaved [element][row][rhs]
  void* mx[2] = {nullptr, nullptr};
  void* mb[2] = {nullptr, nullptr};
  void* mr[2] = {nullptr, nullptr};
  int n[3] = {1, 1, 1};
  // general block-sparse level (cut-cell meshes): task range of every
  // position, task word nbr * 16 + rv * 4 + cv, records cpl[prec] [task][s][s]
  // row-major; transfer to the next coarser level: injection blocks (FP64,
  // FP32) [fine element][s][s], parent of every fine element, children of
  // every coarse element (cptr [nc+1], clist)
  int gen = 0;
  int* tptr = nullptr;
  int* tinfo = nullptr;
  int nbp = 0;                          // padded row count of the column-major dense blocks
  void* gI[2] = {nullptr, nullptr};
  int* gparent = nullptr;
  int* gcptr = nullptr;
  int* gclist = nullptr;
};

// Cut cells of an embedded circle (cutcell.cpp): pieces with their volume
// rules, interface arcs of the cut cells, and the merging of small pieces.
struct CutPiece {
  int i = 0, j = 0, ph = 0;             // host cell, phase (1 inside, 2 outside)
  double area = 0;
  double blo[2] = {0, 0}, bhi[2] = {0, 0};   // bounding box of the piece
  std::vector<double> x, w;             // points [m][2], weights [m]
};
struct CutArc {
  int i = 0, j = 0;
  std::vector<double> x, w, nrm;        // points [m][2], weights, normals [m][2] (out of the circle)
};
struct CutGeometry {
  int n = 0, q = 0;
  double lo[2] = {0, 0}, hi[2] = {1, 1}, h[2] = {1, 1}, c[2] = {0, 0}, r = 0, frac = 0.25;
  bool inside_only = false;             // the disc alone: phase-2 pieces dropped, the circle a boundary
  std::vector<CutPiece> pieces;         // cells in order (x fastest), inside piece first
  std::map<int64_t, int> piece_of;      // ((j n + i) 4 + ph) -> piece
  std::vector<CutArc> arcs;             // one per cut cell, cells in order
  std::vector<int> element;             // piece -> representative piece of its element
  int find(int i, int j, int ph) const {
    auto it = piece_of.find(((int64_t)j * n + i) * 4 + ph);
    return it == piece_of.end() ? -1 : it->second;
  }
};
void build_cut_geometry(CutGeometry& G, int n, const double* lo, const double* hi, double cx, double cy, double r,
                        int q, double frac, bool inside_only = false);
// Gauss rules of the phase-1 and phase-2 parts of the face segment
// {x_axis = fixed, other coordinate in [a, b]}: points [m][2] and weights.
void cut_face_parts(const CutGeometry& G, double a, double b, int axis, double fixed, std::vector<double>* x,
                    std::vector<double>* w);

struct Ctx {
  int device = 0;
  std::string err;
  // problem
  int d = 0, n[3] = {1, 1, 1}, bc[6] = {0};
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  int p = -1, gamma = 0;
  double tau = 0.1, tau0 = -1, c_bdry = 10.0, c_intra = 0.0;
  std::vector<double> mu_vol, mu_if, mu_bf, rho_vol, rho_if;
  // phases (grid-aligned, 1-based) of the finest elements, viscosity per phase,
  // sqrt(mu) diagonal scaling on/off
  std::vector<int> chi;
  std::vector<double> mu_phase;
  int scale_mu = 0;
  double delta = 0.0;
  int nu1 = 1, nu2 = 1, precision = 0;
  // cycle shape: coarse-level visits per level (1 = V-cycle, 2 = W-cycle) and the
  // per-level growth of the smoothing counts (variable V-cycle), capped
  int cyc_gamma = 1, cyc_growth = 1, cyc_cap = 64;
  // smoother colouring of single-phase levels (STK_COLOURS_*)
  int colouring = 0;
  // derived
  int s = 0, nb = 0, q = 0;
  Pattern pat{};
  std::vector<HostLevel> host;
  std::vector<DevLevel> dev;
  bool ready = false;
  // bottom
  int n_snapped = 0;
  int bottom_solver = -1;   // STK_INFO_BOTTOM_SOLVER value of the last setup
  int64_t nbot = 0;
  double* bottom_pinv = nullptr;  // [nbot][nbot]
  double* bot_b64 = nullptr;      // FP64 staging for mixed cycles
  double* bot_x64 = nullptr;
  // transfer matrices P_f (2^d children), [child][s][s] row-major: fine = P coarse
  // index 0: double, 1: float; PT[child][b][a] is the per-child transpose
  void* child_P[2] = {nullptr, nullptr};
  void* child_PT[2] = {nullptr, nullptr};
  // outer-iteration work
  double* r64 = nullptr;
  double* c64 = nullptr;
  double* norm_buf = nullptr;     // device scalars
  double* norm_host = nullptr;    // pinned
  std::atomic<int64_t> launches{0};   // kernels enqueued (calls on one context may come from several threads)
  // graph of one outer iteration, keyed by the caller's x and b pointers
  cudaGraphExec_t graph = nullptr;
  const void* graph_x = nullptr;
  const void* graph_b = nullptr;
  int graph_prec = -1;
  int64_t graph_kernels = 0;
  cudaStream_t stream = nullptr;
  // outer iteration: 0 Richardson, 1 flexible GMRES(restart), 2 flexible GMRES
  // with the Krylov matvec in the cycle precision inside FP64 refinement
  int solver = 0, restart = 30;
  double* kV = nullptr;       // (restart+1) Krylov basis vectors, FP64
  double* kZ = nullptr;       // restart preconditioned vectors, FP64
  double* kw = nullptr;       // work vector
  double* kzero = nullptr;    // zero vector (b of the matvec)
  double* kpart = nullptr;    // multi-dot partials
  double* kdots = nullptr;    // multi-dot results / coefficients (device)
  double* khost = nullptr;    // pinned host staging (dots, coefficients)
  float *kz32 = nullptr, *kw32 = nullptr, *kzero32 = nullptr;   // FP32 matvec of the refined variant
  int kcap = 0;               // restart the buffers were sized for
  // the same for the lockstep FGMRES of several right-hand sides (interleaved vectors)
  double *mkV = nullptr, *mkZ = nullptr, *mkw = nullptr, *mkzero = nullptr, *mkpart = nullptr, *mkdev = nullptr;
  double* mkhost = nullptr;   // pinned staging: dots, coefficients, scales
  float *mkz32 = nullptr, *mkw32 = nullptr, *mkzero32 = nullptr;   // FP32 matvec of the refined variant
  int mk_cap = 0, mk_nr = 0;
  int mrhs_tensor = 1;   // eight right-hand sides with FP32 records: tensor-core kernel
  int df_matvec = 1;     // FGMRES matvec of a low-precision cycle on the FP32 units (double-float)
  // V-cycle alone on the level-0 work vectors, as a CUDA graph
  cudaGraphExec_t cycle_graph = nullptr;
  int cycle_graph_prec = -1;
  int64_t cycle_graph_kernels = 0;
  // element-kernel variant: 0 direct loads, 1 bulk-copy pipeline, 2 warp per element (default),
  // with the pipeline shape per storage precision (CTAs per SM, ring depth)
  int variant_of[4] = {2, 2, 3, 3};   // per storage precision (3: 16-bit records staged)
  int ring_warps[4] = {2, 2, 2, 2};   // warps per element of variant 3
  int launch_overlap = 1;             // element-kernel launches with programmatic serialisation
  int pipe_ctas[4] = {0, 0, 0, 0}, pipe_stages[4] = {0, 0, 0, 0};
  int warp_ctas[4] = {4, 4, 4, 4};   // CTAs (of 8 warps) per SM for the warp-per-element kernel
  // launches of at most this many elements use one CTA per element (latency variant), whatever the variant
  int wide_max = 1024;
  int* dev_err = nullptr;     // raised by a kernel whose bounded wait expired
  // persistent coarse cycle: levels of at most persist_max elements (0: off)
  // run inside one cooperative launch of persist_ctas CTAs per SM
  int persist_max = 0, persist_ctas = 1;
  // the hierarchy stops at the first level below level 0 with at most this
  // many unknowns (0: coarsen until an axis is odd or 2, as Algorithm 1's
  // hierarchy does)
  int64_t bottom_max = 0;
  long long barrier_limit = 2000000000LL;   // clock ticks a grid-barrier wait may take (about 1 s)
  GridBarrierWords* gbar = nullptr;
  int persist_level[4] = {-1, -1, -1, -1};  // first level of the program, per storage precision
  CyclePhase* persist_prog[4] = {nullptr, nullptr, nullptr, nullptr};
  int persist_nphase[4] = {0, 0, 0, 0};
  // element clustering of level 0 (2D, p = 1): requested, and in effect; the
  // cluster level's pattern, host blocks, device records and vectors
  // (cluster layout; ctmp in element layout)
  int cluster_req = 0, cluster_on = 0;
  Pattern cpat{};
  HostLevel chost;
  DevLevel cdev;
  void* cvx[2] = {nullptr, nullptr};
  void* cvb[2] = {nullptr, nullptr};
  void* cvr[2] = {nullptr, nullptr};
  void* ctmp[2] = {nullptr, nullptr};
  // several right-hand sides (interleaved; nr = 4 or 8 once allocated)
  int mr_nr = 0;
  double *mX = nullptr, *mB = nullptr, *mR = nullptr;   // level-0 FP64
  void* mRin = nullptr;                                  // inner right-hand side (cycle precision)
  void* mRb = nullptr;                                   // outer residual in cycle precision
  void* mAcc = nullptr;                                  // accumulated inner correction
  double* mNorm = nullptr;                               // [nr] device, squared norms
  double* mPart = nullptr;
  // learned element-local post-smoother (finest level, low-precision cycles)
  int learn_on = 0, l_in = 0, l_hid = 0, l_ldf = 0;
  float *lW1 = nullptr, *lb1 = nullptr, *lW2 = nullptr, *lb2 = nullptr;   // [in][hid], [hid], [hid][nb], [nb]
  float *lgrad = nullptr, *lm = nullptr, *lv = nullptr;                   // packed like the weights
  int64_t l_nparam = 0;
  int* l_nbr = nullptr;         // natural-order neighbour table of level 0 (l_no slots per element,
  int l_no = 0;                 // the first 2d: -e_0, +e_0, -e_1, ...)
  double* l_ctr = nullptr;      // element centres of a cut-cell level 0 (training fields)
  int* l_ndev = nullptr;        // level-0 grid counts on the device (training fields)
  float *lF = nullptr, *lH = nullptr, *lY = nullptr, *lnrm = nullptr, *lxt = nullptr, *lrt = nullptr;
  double* lsums = nullptr;      // [0] ||r||^2, [1] ||r_t||^2, then partials
  float *lF2 = nullptr, *l_zero = nullptr;   // hidden-layer gradient, zero vector
  float *lTX = nullptr, *lTT = nullptr;   // training residual states [state][element][nb]
  float* lTE = nullptr;         // training error states x* - x [state][element][nb] (supervised objective)
  float* lTg = nullptr;         // MSE targets [element][nb]
  int l_objective = 0;          // 0: ||r - A delta||^2 / ||r||^2, 1: MSE of delta / ||r_i|| against e / ||r_i||
  // outer-iteration acceptance (kappa rule): decisions of the last solve, per
  // outer iteration: -1 plain cycle, 1 correction kept, 0 correction undone
  std::vector<int> l_hist;
  std::vector<double> l_ratio;  // ||r_new|| / (kappa ||r_old||) of each judged iteration
  double l_kappa = 0.0;         // plain contraction of the last solve's first two iterations
  int64_t l_acc = 0, l_rej = 0; // totals since stk_learn_enable
  cudaGraphExec_t lgraph = nullptr, rgraph = nullptr;   // learned iteration, undo
  const void* lgraph_x = nullptr;
  const void* lgraph_b = nullptr;
  int64_t lgraph_kernels = 0, rgraph_kernels = 0;
  int64_t l_rows = 0, l_cap = 0;
  int l_adam_t = 0;
  cudaGraphExec_t mgraph = nullptr;
  int mgraph_key[3] = {-1, -1, -1};                      // nr, inner, precision
  int64_t mgraph_kernels = 0;
  std::vector<void*> allocations;
  int64_t device_bytes = 0;   // bytes the library allocated for this context
  // embedded circle (cut-cell mesh of the box): centre, radius, merge
  // fraction; density per phase and delta of an unsteady cut-cell problem;
  // the geometry (built on demand for the current mesh and degree)
  int cut = 0;
  double cut_c[2] = {0, 0}, cut_r = 0, cut_frac = 0.25;
  int cut_inside = 0;           // one phase: the disc inside the circle, Dirichlet on the circle
  std::vector<double> rho_phase;
  double cut_delta = 0.0;
  int gen_warps = 0;                    // warps per element of the general element kernel (0: by launch size)
  std::shared_ptr<CutGeometry> cutg;
  std::shared_ptr<struct CutState> cuts;   // elements, faces and finest operators after setup
};

// ---- setup.cpp --------------------------------------------------------------
void build_pattern(int d, int p, int gamma, bool multiphase, Pattern& pat);
void greedy_colours(const Ctx& c, const int* n, std::vector<int>& colour);
int assemble_rhs_host2(const Ctx& c, const double* f_vol, const double* bdata, const double* idata, double* b);
void interface_info(const Ctx& c, std::vector<int>& chim, std::vector<int>& chip, std::vector<double>& nrm);
int setup_host(Ctx& c);                    // fine assembly, coarsening, Stokes blocks
void child_matrices(int d, int p, std::vector<double>& out);   // [2^d][s][s]
void gauss_rule(int q, std::vector<double>& x, std::vector<double>& w);
int invert_blocks(int n, int count, const double* A, double* Ainv, std::string& err);
int pseudo_inverse_sym(int n, std::vector<double>& A, std::vector<double>& pinv, int& snapped, double theta);
// Equilibration of a symmetric matrix for the bottom eigensolvers:
// S_i = (row 1-norm)^(-1/2), Ah = S A S.
void equilibrate_sym(int n, const std::vector<double>& A, std::vector<double>& S, std::vector<double>& Ah);
// pinv <- P pinv P with P the orthogonal projector off the span of the nk rows
// of K (row-major nk x n, orthonormalised here); pinv symmetric n x n.
void project_off_kernel(int n, std::vector<double>& pinv, std::vector<double>& K, int nk);
int pseudo_inverse_jacobi(int n, std::vector<double>& A, std::vector<double>& pinv, int& snapped,
                          double theta);
void element_index(const int* n, int d, int64_t e, int* idx);
void face_points(const Ctx& c, int kind, std::vector<double>& xyz, std::vector<double>* nrm);
int assemble_rhs_host(const Ctx& c, const double* f_vol, const double* bdata, double* b);
int build_cluster_level(const Ctx& c, const HostLevel& H, const Pattern& ep, const Pattern& cp, HostLevel& HC,
                        std::string& err);
void psi_eval(int p, double x, double* v, double* dv);
void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& fn);

// ---- cutsetup.cpp -------------------------------------------------------------
const CutGeometry& cut_geometry(Ctx& c);    // (re)built for the current mesh and degree
int setup_cut(Ctx& c, std::string& err);     // levels of the cut-cell hierarchy (general block-sparse)
int64_t cut_count_points(Ctx& c, int kind);
void cut_points(Ctx& c, int kind, std::vector<double>& xyz, std::vector<double>* nrm, std::vector<int>* phase);
int cut_assemble_rhs(Ctx& c, const double* f_vol, const double* bdata, const double* idata, double* b,
                     std::string& err);
// Level-0 element neighbours across the four faces of each element's anchor
// cell in its own phase ([ne][4]: -x, +x, -y, +y; -1 none) and element box
// centres in box-relative coordinates ([ne][2]).
void cut_face_neighbours(Ctx& c, std::vector<int>& nbr, std::vector<double>& ctr);


// ---- kernels.cu / learn.cu launchers ------------------------------------------
constexpr int MODE_GS = 0, MODE_RESID = 1;   // element kernel: colour step, or residual
cudaError_t launch_element(const Pattern& pat, int storage, int mode, int pos0, int npos,
                           const int* perm, const int* nbr, const void* cpl, const void* mat,
                           const void* b, void* x, void* r, cudaStream_t st);
cudaError_t launch_restrict(int vec64, int d, int s, int nb, const int* nc, const int* nf, int64_t nec,
                            const void* P, const void* r, void* rc, cudaStream_t st);
cudaError_t launch_prolong(int vec64, int d, int s, int nb, const int* nf, const int* nc, int64_t nec,
                           const void* PT, const void* xc, void* x, cudaStream_t st);
cudaError_t launch_bottom(int vec64, int64_t n, const double* pinv, const void* b, void* x,
                          cudaStream_t st);
cudaError_t launch_axpy(int y64, int x64, int64_t n, void* y, const void* x, cudaStream_t st);
cudaError_t launch_convert(int y64, int x64, int64_t n, void* y, const void* x, cudaStream_t st);
cudaError_t launch_to_bf16(int64_t n, void* y, const double* x, cudaStream_t st);
cudaError_t launch_sumsq(int64_t n, const double* x, double* part, double* out, cudaStream_t st);
cudaError_t launch_multidot(int64_t n, int k, const double* V, int64_t ldv, const double* w, double* part,
                            double* out, cudaStream_t st);
cudaError_t launch_multiaxpy(int64_t n, int k, double alpha, const double* coef, const double* V, int64_t ldv,
                             double* w, cudaStream_t st);
cudaError_t launch_scale(int64_t n, double s, const double* x, double* y, cudaStream_t st);
cudaError_t launch_element_pipe(const Pattern& pat, int storage, int mode, int pos0, int npos, const int* perm,
                                const int* nbr, const void* cpl, const void* mat, const void* b, void* x, void* r,
                                int* err, int ctas, int stages, cudaStream_t st);
void prepare_pipe_kernels();
void prepare_mrhs_kernels();
cudaError_t launch_element_mrhs(const Pattern& pat, int storage, int nr, int mode, int pos0, int npos,
                                const int* perm, const int* nbr, const void* cpl, const void* mat, const void* b,
                                void* x, void* r, cudaStream_t st, int tensor = 0, int tensor_small = 0);
cudaError_t launch_restrict_mr(int vec64, int d, int s, int nb, int nr, const int* nc, const int* nf, int64_t nec,
                               const void* P, const void* r, void* rc, cudaStream_t st);
cudaError_t launch_prolong_mr(int vec64, int d, int s, int nb, int nr, const int* nf, const int* nc, int64_t nec,
                              const void* PT, const void* xc, void* x, cudaStream_t st);
cudaError_t launch_bottom_mr(int vec64, int64_t n, int nr, const double* pinv, const void* b, void* x, cudaStream_t st);
cudaError_t launch_interleave(int kind, int64_t m, int nr, int nq, int to_interleaved, void* out, const void* in,
                              cudaStream_t st);
cudaError_t launch_sumsq_mr(int64_t m, int nr, const double* x, double* part, double* out, cudaStream_t st);
cudaError_t launch_multidot_mr(int64_t n, int nr, int k, const double* V, int64_t ldv, const double* w,
                               double* part, double* out, cudaStream_t st);
cudaError_t launch_multiaxpy_mr(int64_t n, int nr, int k, double alpha, const double* coef, const double* V,
                                int64_t ldv, double* w, cudaStream_t st);
cudaError_t launch_scale_mr(int64_t n, int nr, const double* s, const double* x, double* y, cudaStream_t st);
cudaError_t launch_features(int ne, int nb, int nface, int NO, int ldf, const int* nbr_nat, const float* r, float* F,
                            float* nrm, cudaStream_t st);
cudaError_t launch_sgemm(int M, int N, int K, int ta, int tb, const float* A, int lda, const float* B, int ldb,
                         float* C, int ldc, const float* bias, int act, float alpha, float beta, cudaStream_t st);
cudaError_t launch_colsum(int M, int N, const float* A, int lda, float* out, float alpha, cudaStream_t st);
cudaError_t launch_fill(double* v, double a, cudaStream_t st);
cudaError_t launch_mse_grad(int64_t n, float scale, const float* Y, const float* T, float* dY, double* part,
                            double* out, cudaStream_t st);
cudaError_t launch_tanh_back(int64_t n, const float* H, float* dH, cudaStream_t st);
cudaError_t launch_adam(int64_t n, float lr, float b1, float b2, float c1, float c2, float eps, float* w,
                        const float* g, float* m, float* v, cudaStream_t st);
cudaError_t launch_apply_correction(int ne, int nb, int ldy, const float* x, const float* nrm, const float* Y, float* xt,
                                    cudaStream_t st);
cudaError_t launch_sumsq_f(int64_t n, const float* x, double* part, double* out, cudaStream_t st);
cudaError_t launch_smooth_field(int ne, int nb, int s, int d, const int* n_dev, const double* ctr, uint64_t seed,
                                float* x,
                                cudaStream_t st);
cudaError_t launch_target(int ne, int nb, int ldt, const float* xs, const float* x, const float* nrm, float* T,
                          cudaStream_t st);
cudaError_t launch_scale_f(int64_t n, float a, const float* x, float* y, cudaStream_t st);
cudaError_t launch_scale_by_norm(int64_t n, const double* sums, float* g, cudaStream_t st);
cudaError_t launch_element_wide(const Pattern& pat, int storage, int mode, int pos0, int npos, const int* perm,
                                const int* nbr, const void* cpl, const void* mat, const float* tsc, const float* rsc,
                                const void* b, void* x, void* r, cudaStream_t st, int overlap = 0);
cudaError_t launch_element_df(const Pattern& pat, int pos0, int npos, const int* perm, const int* nbr,
                              const void* cpl_hi, const void* cpl_lo, const void* dia_hi, const void* dia_lo,
                              const float* z, double* w, int ctas, cudaStream_t st);
cudaError_t launch_fp32_remainder(int64_t n, const double* a, void* lo, cudaStream_t st);
void prepare_df_kernels();
cudaError_t launch_to_fp16_tasks(int64_t npos, int S, int T, int TRP, void* dst, float* tsc, const double* src,
                                 cudaStream_t st);
cudaError_t launch_to_fp16_rows(int64_t npos, int nb, int NBP, void* dst, float* rsc, const double* src,
                                cudaStream_t st);
cudaError_t launch_element_warp(const Pattern& pat, int storage, int mode, int pos0, int npos, const int* perm,
                                const int* nbr, const void* cpl, const void* mat, const float* tsc, const float* rsc,
                                const void* b, void* x, void* r, int ctas, cudaStream_t st, int overlap = 0);
cudaError_t launch_element_ring(const Pattern& pat, int storage, int warps, int mode, int pos0, int npos,
                                const int* perm, const int* nbr, const void* cpl, const void* mat, const float* tsc,
                                const float* rsc, const void* b, void* x, void* r, int overlap, cudaStream_t st);
void pipe_default_shape(const Pattern& pat, int storage, int* ctas, int* stages);

cudaError_t launch_fp64_fma(int blocks, int iters, double* out, cudaStream_t st);
cudaError_t launch_cluster_permute(int vec64, int n0, int n1, int s, int nvar, int to_cluster, const void* in,
                                   void* out, cudaStream_t st);
cudaError_t launch_coarse_cycle(const Pattern& pat, int storage, const CyclePhase* phases, int nphase,
                                GridBarrierWords* gb, int* err, long long limit, int grid, cudaStream_t st);
cudaError_t launch_batch_solve(const BatchProblem* probs, int nprob, const BatchStep* steps, int nsteps,
                               const BatchTask* tasks, int maxit, double rtol, int smax, size_t smem,
                               GridBarrierWords* gb, int* err, long long limit, int grid, cudaStream_t st);
size_t batch_smem_bytes(const Pattern& pat);
cudaError_t launch_gen_element(int storage, int mode, int warps, int s, int nb, int nbp, int pos0, int npos,
                               const int* perm, const int* tptr, const int* tinfo, const void* cpl, const void* mat,
                               const void* b, void* x, void* r, cudaStream_t st, int overlap = 0);
cudaError_t launch_gen_restrict(int vec64, int nc, int s, int nb, const int* cptr, const int* clist, const void* I,
                                const void* r, void* rc, cudaStream_t st);
cudaError_t launch_gen_prolong(int vec64, int nf, int s, int nb, const int* parent, const void* I, const void* xc,
                               void* x, cudaStream_t st);
cudaError_t launch_barrier_selftest(GridBarrierWords* gb, int* err, long long limit, int rounds, int absent, int grid,
                                    unsigned int* passed, cudaStream_t st);

// ---- api.cu -------------------------------------------------------------------
// One element-kernel launch (colour step in MODE_GS, residual in MODE_RESID) on
// level l of c, on the kernel variant the context's tuning picks for it.
cudaError_t run_element(Ctx& c, int l, int prec, int mode, int pos0, int npos, const void* mat, const void* b,
                        void* x, void* r, cudaStream_t st);
cudaError_t run_element_on(Ctx& c, const Pattern& pat, DevLevel& D, int prec, int mode, int pos0, int npos,
                           const void* mat, const void* b, void* x, void* r, cudaStream_t st);

}  // namespace stk

// The opaque handle of the C ABI is the library context.
struct stk_ctx : public stk::Ctx {};
