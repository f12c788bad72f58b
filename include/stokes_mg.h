/*
 * stokes_mg.h -- C ABI of the GB300 multigrid library for LDG-discretised
 * Stokes systems (Saye, "Fast multigrid solution of high-order accurate
 * multi-phase Stokes problems", arXiv:1911.05888).
 *
 * The library builds, for a Cartesian mesh, the LDG operator of the paper's
 * eq. (blockform) / (timedep2) on every level of a geometric hierarchy
 * (operator coarsening, Appendix B, Algorithms 2 and 3), factorises the
 * element blocks, and runs on one GPU the V-cycle of Algorithm 1: coloured
 * element block Gauss-Seidel, residual, restriction by (I_2h^h)^T,
 * prolongation by injection and a pseudo-inverse bottom solve.
 *
 * Conventions
 *  - Every call returns an int status: STK_OK (0) or a negative STK_ERR_*.
 *    stk_last_error(ctx) gives a message owned by ctx, valid until the next
 *    call on ctx.  No C++ exception crosses this interface.
 *  - Host arrays passed in are owned by the caller and only read during the
 *    call.  Device pointers (suffix _dev) are caller-owned device memory on
 *    the context's device; the library never frees them.  Streams are
 *    cudaStream_t passed as void* (NULL = legacy default stream).
 *  - The library owns its hierarchy, work vectors and CUDA graphs until
 *    stk_destroy.
 *  - Vectors are element-blocked: [element][nb] with nb = (d+1) (p+1)^d,
 *    the per-element order [u_1 modes, ..., u_d modes, p modes], modes
 *    lexicographic with the x index fastest, elements lexicographic with x
 *    fastest.  The basis is the tensor product of sqrt(2l+1) P_l (Legendre) on
 *    each element's reference cube, so the element mass matrix is |E| times
 *    the identity.
 *  - Values are double unless stated.  With nrhs > 1 a vector is
 *    [nrhs][element][nb] (right-hand sides outermost).
 */
#ifndef STOKES_MG_H
#define STOKES_MG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  STK_OK = 0,
  STK_ERR_INVALID_ARG = -1,
  STK_ERR_OOM = -2,
  STK_ERR_SINGULAR_BLOCK = -3,
  STK_ERR_TIMEOUT = -4,
  STK_ERR_DIVERGED = -5,
  STK_ERR_NOT_SETUP = -6,
  STK_ERR_CUDA = -7
};

/* Boundary types of a box side (governing eq. (govern3) of the paper). */
enum { STK_BC_PERIODIC = 0, STK_BC_DIRICHLET = 1, STK_BC_STRESS = 2 };

/* Storage precision of the element blocks inside the V-cycle. */
enum { STK_FP64 = 0, STK_FP32 = 1, STK_BF16 = 2, STK_FP16 = 3 };

/* Point sets at which the caller samples coefficients and data. */
enum { STK_PTS_VOLUME = 0, STK_PTS_INTERIOR_FACE = 1, STK_PTS_BOUNDARY_FACE = 2, STK_PTS_INTERFACE = 3 };

typedef struct stk_ctx stk_ctx;

/* Create a context on CUDA device `device`.  *out is set on success. */
int stk_create(stk_ctx** out, int device);
/* Release everything the context owns.  NULL is accepted. */
int stk_destroy(stk_ctx* ctx);
/* Message describing the last error on ctx (never NULL). */
const char* stk_last_error(stk_ctx* ctx);

/*
 * Mesh: the box [lo, hi] in d = 2 or 3 dimensions split into n[0] x ... x
 * n[d-1] equal elements (Section 2: Cartesian grids).  bc[2k] is the type of
 * the low side of axis k, bc[2k+1] of the high side; STK_BC_PERIODIC must be
 * set on both sides of an axis.
 */
int stk_set_mesh(stk_ctx* ctx, int d, const int* n, const double* lo, const double* hi,
                 const int* bc);

/*
 * Discretisation (Section 2): degree p >= 1 of the tensor-product space Q_p
 * for velocity and pressure; gamma = 0 standard form, 1 viscous-stress form
 * (eq. govern1).  Quadrature: Gauss with 2p+2 points per axis for the
 * mu/rho-weighted mass matrices, face means and data integrals.
 */
int stk_set_discretisation(stk_ctx* ctx, int p, int gamma);

/*
 * Penalty parameters (Section 4 and Appendix A.1): tau is the pressure
 * penalty prefactor of eq. (taueqn), tau_p = tau h / mu; tau0 the prefactor
 * of the vanishing-viscosity limit in eq. (taupgeneral).  The velocity
 * penalties are tau_u,bdry = c_bdry p mu / h on Dirichlet faces and
 * tau_u,0 = c_intra p mu / h on interior faces (Cartesian default 10 and 0).
 */
int stk_set_penalty(stk_ctx* ctx, double tau, double tau0, double c_bdry, double c_intra);

/* Number of sample points of a point set (after stk_set_mesh and
 * stk_set_discretisation): volume Gauss points [element][q^d], interior-face
 * points [face][q^(d-1)], boundary-face points [face][q^(d-1)] with q = 2p+2.
 * Faces are enumerated axis by axis; interior faces by their right element
 * in element order (periodic wrap faces included), boundary faces by
 * (axis, low side then high side, element order). */
int stk_num_points(stk_ctx* ctx, int kind, int64_t* count);
/* Coordinates [count][d] of a point set, and for boundary faces the outward
 * unit normals [count][d] (normals may be NULL). */
int stk_get_points(stk_ctx* ctx, int kind, double* xyz, double* normals);

/*
 * Viscosity mu > 0 sampled at the volume, interior-face and boundary-face
 * points (eq. sigmaresult: M_mu; face values enter the penalties as face
 * means).  Checked: every value finite and positive.
 */
int stk_set_viscosity(stk_ctx* ctx, const double* mu_vol, const double* mu_iface,
                      const double* mu_bface);

/*
 * Unsteady problem (eq. timedep1/timedep2): density rho > 0 at the volume and
 * interior-face points and the parameter delta > 0 (proportional to the time
 * step).  The pressure penalty follows eq. (taupgeneral) and is coarsened by
 * Algorithm 3.  delta = 0 returns to the steady problem.
 */
int stk_set_density(stk_ctx* ctx, const double* rho_vol, const double* rho_iface, double delta);

/*
 * V-cycle options (Algorithm 1): nu1 pre- and nu2 post-smoothing sweeps of
 * the coloured block Gauss-Seidel method; precision = STK_FP64 (plain) or
 * STK_FP32 / STK_BF16 / STK_FP16 (element blocks stored in that type and
 * accumulated in FP32 inside the cycle; the outer residual and the bottom
 * solve stay FP64).  STK_FP16 blocks carry a power-of-two scale per s x s
 * coupling sub-block and per row of A_ii^{-1} and A_ii (the group's largest
 * magnitude scaled into [2^14, 2^15), entries rounded to nearest even from
 * FP64), so FP16's 11-bit significand holds over the blocks' whole range.
 * Several right-hand sides (stk_solve_multi) and element-kernel variants 0
 * and 1 take FP64, FP32 or BF16 blocks only.  Errors: STK_ERR_INVALID_ARG.
 */
int stk_set_cycle(stk_ctx* ctx, int nu1, int nu2, int precision);

/*
 * Cycle shape (Section 6 names W-cycles and variable V-cycles as the
 * alternatives to Algorithm 1's V-cycle).  gamma = visits of level l+1 per
 * visit of level l (1: V-cycle, 2: W-cycle, 3); the coarse correction starts
 * from zero and each further visit continues from the previous visit's
 * result; the coarsest level is solved exactly and visited once.  Smoothing
 * on level l takes min(nu * growth^l, max(nu, max_sweeps)) sweeps for
 * nu = nu1 and nu = nu2 (growth 1: fixed counts; growth 2: the variable
 * V-cycle).  Defaults 1, 1, 64.  Applies to every cycle of the context
 * (single and several right-hand sides).  Errors: STK_ERR_INVALID_ARG
 * unless 1 <= gamma <= 3, 1 <= growth <= 4, 1 <= max_sweeps <= 256.
 */
int stk_set_cycle_shape(stk_ctx* ctx, int gamma, int growth, int max_sweeps);

/*
 * Colouring of the block Gauss-Seidel sweep on single-phase levels (Section 3:
 * the elements of one colour are updated together, so no two of them may
 * couple).  STK_COLOURS_AUTO (default): the checkerboard (i_1+...+i_d) mod 2
 * for the standard form (gamma = 0), whose operator couples face neighbours
 * only, and the 2^d parity colours sum_k (i_k mod 2) 2^k for the
 * viscous-stress form, whose diagonal (2D) / edge (3D) couplings the
 * checkerboard would not separate.  STK_COLOURS_PARITY forces the 2^d colours;
 * STK_COLOURS_CHECKERBOARD forces two colours (stk_setup then returns
 * STK_ERR_INVALID_ARG unless gamma = 0 and the problem has one phase).  Problems
 * with phases always take the greedy colouring.  Takes effect at the next
 * stk_setup.  Errors: STK_ERR_INVALID_ARG for an unknown mode.
 */
/*
 * Persistent coarse cycle (not in the paper; Algorithm 1 unchanged): every
 * level below level 0 with at most max_elements elements, from the first
 * such level down to the bottom and back (its colour steps, residual,
 * restriction with the coarse iterate zeroed, coarse visits of the cycle
 * shape, bottom solve, prolongation), runs as ONE cooperative launch of
 * ctas_per_sm CTAs per SM that walks a phase program built at setup, with a
 * grid barrier between phases.  Each phase runs the same per-element code as
 * the kernel it replaces, so iterates are unchanged bit for bit.  Every
 * barrier wait is bounded (about a second of clock ticks); on expiry the
 * launch sets the context's error word and returns, and the solve reports
 * STK_ERR_TIMEOUT.  max_elements = 0 (the default) turns it off.  Errors:
 * STK_ERR_INVALID_ARG unless max_elements >= 0 and 1 <= ctas_per_sm <= 8.
 */
int stk_set_persistent(stk_ctx* ctx, int max_elements, int ctas_per_sm);
/*
 * Element clustering (the Concluding Remarks' suggestion for p = 1): on = 1
 * makes the block Gauss-Seidel smoother of level 0 use clusters of 2 x 2
 * elements (the children of one cell of level 1) as its blocks: x_C <-
 * A_CC^{-1}(b_C - sum_{D != C} A_CD x_D), clusters coloured like elements
 * (checkerboard of the cluster grid for the standard form, 2^d parity
 * colours otherwise).  Applies at the next stk_setup to 2D problems of degree
 * 1 with one phase whose periodic axes have an even number of clusters
 * (STK_INFO_CLUSTERS tells whether it took effect); cycles of one
 * right-hand side only (stk_solve_multi keeps element blocks, and
 * stk_solve_batch_persistent refuses such contexts).  The cluster blocks are
 * 48 x 48 and run on the element kernels; vectors move between element and
 * cluster layout at the cycle's start and end and around the transfers.
 * Errors: STK_ERR_INVALID_ARG unless on is 0 or 1.
 */
int stk_set_clusters(stk_ctx* ctx, int on);
/*
 * Earlier bottom level (Section 3 leaves the depth of the hierarchy open;
 * Algorithm 1 only needs an exact coarsest solve): the hierarchy stops at the
 * first level below level 0 with at most max_unknowns unknowns, which is then
 * solved by the dense eigen pseudo-inverse (cuSOLVER above 1200 unknowns).
 * 0 (default): coarsen while every n_k is even and above 2 (cut-cell
 * meshes: until the grid is 2 x 2).  Takes effect at the next stk_setup.
 * Errors: STK_ERR_INVALID_ARG outside 0..20000.
 */
int stk_set_bottom(stk_ctx* ctx, int64_t max_unknowns);
/*
 * Self-test of the bounded grid barrier (a diagnostic, no solver state is
 * touched): a cooperative launch of the persistent cycle's grid passes four
 * barriers; with absent >= 0 that CTA returns at once and never arrives, so
 * every other CTA must give up after limit_ticks clock ticks
 * (1e3 <= limit_ticks <= 4e9).  *passed = barrier passages counted (CTAs x
 * barriers passed).  Returns STK_OK when all barriers completed,
 * STK_ERR_TIMEOUT when the bound expired; the context stays usable either way.
 */
int stk_barrier_selftest(stk_ctx* ctx, int absent, int64_t limit_ticks, int64_t* passed);

#define STK_COLOURS_AUTO 0
#define STK_COLOURS_PARITY 1
#define STK_COLOURS_CHECKERBOARD 2
int stk_set_colouring(stk_ctx* ctx, int mode);

/*
 * Setup: fine-level LDG assembly (Appendix A), operator coarsening
 * (Algorithm 2, or 3 when unsteady) down to the bottom level (some n_k odd or
 * equal to 2), the Stokes blocks of every level, element-block inverses (FP64
 * Gauss-Jordan with partial pivoting; STK_ERR_SINGULAR_BLOCK if a pivot
 * vanishes), the parity colouring, and the bottom pseudo-inverse (symmetric
 * eigendecomposition with |lambda| <= 1e-10 max|lambda| snapped to zero).
 * Allocates all device memory the cycle needs.
 */
int stk_setup(stk_ctx* ctx, void* stream);

/*
 * Hierarchy sizes: number of levels, elements per level (array of
 * nlevels entries, may be NULL), block size nb, number of snapped bottom
 * eigenvalues (may be NULL).
 */
int stk_get_sizes(stk_ctx* ctx, int* nlevels, int64_t* n_elements, int* nb, int* n_snapped);

/*
 * Introspection of a context (not a step of the method): *value receives
 *   STK_INFO_BOTTOM_SOLVER   eigensolver of the last setup's bottom pseudo-
 *                            inverse (Section 3 footnote): 0 cyclic Jacobi
 *                            (host, <= 300 unknowns), 1 equilibrated
 *                            Householder + implicit QR (host, <= 1200),
 *                            2 equilibrated cuSOLVER syevd (device, above);
 *   STK_INFO_BOTTOM_UNKNOWNS unknowns of the bottom level;
 *   STK_INFO_COLOURS         colours of the level-0 smoother;
 *   STK_INFO_DEVICE_BYTES    device bytes the library holds for the context;
 *   STK_INFO_CLUSTERS        1 when level 0 smooths element clusters;
 *   STK_INFO_COUPLING_BLOCKS s x s coupling sub-blocks level 0 stores (the
 *                            records a colour sweep streams besides the
 *                            dense A_ii^{-1}).
 * All but STK_INFO_DEVICE_BYTES need stk_setup (else STK_ERR_NOT_SETUP); an unknown key is
 * STK_ERR_INVALID_ARG.
 */
#define STK_INFO_BOTTOM_SOLVER 0
#define STK_INFO_BOTTOM_UNKNOWNS 1
#define STK_INFO_COLOURS 2
#define STK_INFO_DEVICE_BYTES 3
#define STK_INFO_CLUSTERS 4
#define STK_INFO_COUPLING_BLOCKS 5
int stk_get_info(stk_ctx* ctx, int what, int64_t* value);

/* Dense nb x nb block A_ij (row element i, column element j, natural
 * element indices) of the level-`level` operator, row-major, into a host
 * array; zero when the elements do not couple. */
int stk_get_block(stk_ctx* ctx, int level, int64_t i, int64_t j, double* out);

/* Right-hand side b (Appendix A, eq. appstokes1/appstokes2 multiplied by M)
 * from samples: f_vol [volume point][d+1] = (f_1..f_d, fdiv) with
 * -div u = fdiv; bdata [boundary-face point][d] = Dirichlet velocity g on
 * Dirichlet faces, stress sigma.n = h on stress faces (ignored on periodic
 * sides).  Writes the host array b [element][nb]. */
int stk_assemble_rhs(stk_ctx* ctx, const double* f_vol, const double* bdata, double* b);

/*
 * Phases (Section 5.6 and Appendix A): chi [element] in 1..nphase gives the
 * phase of each finest element (interfaces along element faces), mu_phase
 * [nphase] the viscosity of each phase.  Interphase faces get the
 * viscosity-upwinded fluxes of eq. (viscosityupwind) with lambda = 0, 1/2, 1,
 * the penalty tau_ij = 3 p min(mu-, mu+) / h and no pressure penalty; coarse
 * levels agglomerate only same-phase children (the hierarchy ends at the
 * first level where a coarse cell would mix phases); smoothing uses a greedy
 * colouring (elements in order, smallest colour unused within the coupling
 * stencil).  scale = 1 replaces every level's operator by D A D with D =
 * mu_E^{-1/2} on velocity and mu_E^{1/2} on pressure unknowns (mu_E the
 * element mean of mu); every call then works on that scaled system
 * (b~ = D b, x = D x~; stk_get_scaling gives D).  nphase = 0 clears phases.
 * Call after stk_set_discretisation and before stk_setup.
 */
int stk_set_phases(stk_ctx* ctx, int nphase, const int* chi, const double* mu_phase, int scale);
/* For every interior-face point: the phase of the - and + element of an
 * interphase face (0 and 0 on faces inside one phase) and the face normal
 * [point][d] (from the lower phase into the higher on interphase faces). */
int stk_get_interface(stk_ctx* ctx, int* chi_minus, int* chi_plus, double* normals);
/* stk_assemble_rhs with interface jump data: idata [interior-face
 * point][2d] = (g_ij, h_ij) with g_ij = u(-) - u(+) and h_ij = sigma(-) n -
 * sigma(+) n on interphase faces (ignored elsewhere; may be NULL without
 * phases).  b is the right-hand side of the unscaled system. */
int stk_assemble_rhs2(stk_ctx* ctx, const double* f_vol, const double* bdata, const double* idata, double* b);
/* Colour of every element (natural order) on a smoothing level. */
int stk_get_colours(stk_ctx* ctx, int level, int* colours);
/* Level-0 diagonal scaling D [element][nb] (all ones without scaling). */
int stk_get_scaling(stk_ctx* ctx, double* D);

/* ---- hot path ------------------------------------------------------------ */

/* r = b - A x on level 0 in FP64 (eq. blockform); optional ||r||_2 into
 * *norm_out (host; synchronises the stream when non-NULL). */
int stk_residual(stk_ctx* ctx, const double* x_dev, const double* b_dev, double* r_dev,
                 double* norm_out, void* stream);

/* One colour step of the block Gauss-Seidel smoother on level `level` in
 * FP64: every element i of colour c (parity colouring sum_k (i_k mod 2) 2^k,
 * or the greedy colouring with phases; stk_get_colours) gets
 * x_i = A_ii^{-1} (b_i - sum_{j != i} A_ij x_j) (Section 3). */
int stk_gs_colour(stk_ctx* ctx, int level, int colour, double* x_dev, const double* b_dev,
                  void* stream);

/* The colour step of stk_gs_colour and the residual of Algorithm 1
 * on any smoothing level with the blocks stored in `precision`: STK_FP64
 * (x, b, r are double) or the precision given to stk_set_cycle before
 * stk_setup (x, b, r are float, accumulation in FP32).  These run the same
 * kernels as the V-cycle; they exist so callers can time and test them. */
int stk_gs_colour_ex(stk_ctx* ctx, int level, int colour, int precision, void* x_dev,
                     const void* b_dev, void* stream);
int stk_residual_ex(stk_ctx* ctx, int level, int precision, const void* x_dev, const void* b_dev,
                    void* r_dev, void* stream);

/* One V-cycle of Algorithm 1 in place on level 0 in FP64: x <- V(x, b). */
int stk_vcycle(stk_ctx* ctx, double* x_dev, const double* b_dev, void* stream);

/* Restriction r_c = (I_2h^h)^T r (level -> level+1) and prolongation
 * x += I_2h^h x_c (level+1 -> level), FP64 (the transfers of Algorithm 1). */
int stk_restrict(stk_ctx* ctx, int level, const double* r_dev, double* rc_dev, void* stream);
int stk_prolong(stk_ctx* ctx, int level, const double* xc_dev, double* x_dev, void* stream);
/*
 * The bottom solver's least-squares (Moore-Penrose) inverse on the host
 * (Section 3 footnote) of the symmetric n x n matrix A (row-major host array,
 * caller-owned, not modified; its symmetric part is used).  A is equilibrated
 * to A^ = S A S (S_i = row 1-norm^(-1/2)); the eigenvalues of A^ with
 * |lambda| <= theta max|lambda| are snapped to zero (Householder reduction to
 * tridiagonal form, shifted implicit QR; cyclic Jacobi if that does not
 * converge), and the result is projected off the kernel of A.  pinv:
 * caller-owned host array n x n; *snapped (may be NULL) = eigenvalues set to
 * zero.  Needs no device; stk_setup uses it for bottom levels of 301 to 1200
 * unknowns.  Errors: STK_ERR_INVALID_ARG (n outside 1..20000, NULL arrays,
 * theta outside [0,1)), STK_ERR_OOM.
 */
int stk_host_pseudo_inverse(int n, const double* A, double theta, double* pinv, int* snapped);

/*
 * Cut cells of an embedded circle (Section 5's circular interface; host only,
 * no context or device needed): the n x n grid on [lo, hi] (2 entries each)
 * cut by the circle of centre (cx, cy) and radius r.  Quadrature by dimension
 * reduction with q Gauss points per sub-interval (height direction per cell
 * along the larger normal component; chords found analytically); pieces below
 * merge_fraction of their cell join the same-phase piece across the cell face
 * they share most with (among neighbours not small themselves); the merged
 * elements are coloured greedily (elements in the order of their
 * representative piece, smallest colour not used by an element reachable
 * through the coupling stencil {|o| <= 1} U {+-2 e_k} of any host cell).
 * Pieces: every uncut cell, and the inside (phase 1) and outside (phase 2)
 * parts of every cut cell, ordered by cell (x fastest), inside first.
 * *npieces: in, the capacity of the output arrays; out, the number of pieces
 * (call with capacity 0 to size them).  Outputs (may be NULL): cell [np][2],
 * phase [np], area [np], element [np] (the representative piece of the
 * element the piece belongs to), colour [np] (of its element),
 * *interface_length (the interface rule's total weight).  A context solves
 * on these elements after stk_set_levelset_circle.  Errors:
 * STK_ERR_INVALID_ARG (n outside 1..4096, r <= 0, q outside 1..32, empty box).
 */
int stk_cut_cells(int n, const double* lo, const double* hi, double cx, double cy, double r, int q,
                  double merge_fraction, int64_t* npieces, int* cell, int* phase, double* area, int* element,
                  int* colour, double* interface_length);

/*
 * Embedded circle (Section 5's curved interface; the multi-phase problems of
 * Section 6): the 2D n x n mesh of stk_set_mesh (square cells, Dirichlet on
 * every side) is cut by the circle of centre (cx, cy) and radius r into
 * phase 1 (inside) and phase 2 (outside).  The cells' pieces carry the
 * quadrature of stk_cut_cells with q = 2p + 2 points per sub-interval, pieces
 * below a quarter of their cell are merged (stk_cut_cells with merge fraction
 * 0.25), and each merged element takes the tensor Legendre basis Q_p on its
 * bounding box (the union of its host cells), so element mass matrices are
 * dense and vectors stay [element][nb] with elements in the order of their
 * representative piece.  stk_setup then assembles Appendix A on these
 * elements: intraphase lifts into the right element with the pressure
 * penalty tau h / mu (eq. eop; eq. taupgeneral with densities), Dirichlet
 * penalty c_bdry p mu / h, and on the circle the viscosity-upwinded fluxes of
 * eq. (viscosityupwind) with the penalty 3 p min(mu-, mu+) / h.  The
 * hierarchy agglomerates the elements of every level by the parent cell of
 * their anchor cell and by phase until the grid is 2 x 2; a coarse element's
 * basis lives on its members' union box, the injection onto a member f is the
 * L2 projection M_f^{-1} int_f phi_f phi_c^T, and the coarse operators follow
 * Algorithm 2 (Algorithm 3 with densities).  The smoother colours every level
 * greedily (elements in order, smallest colour not used by an element within
 * two face / interface steps; on coarse levels by an element holding coupled
 * members).  Needs stk_set_phases(ctx, 2, NULL, mu_phase, scale), or
 * stk_set_phases(ctx, 1, NULL, &mu, scale) for the disc alone (Section 5's
 * curved domain: the outside pieces are dropped and the circle carries
 * Dirichlet data, lifted with its outward normal and penalised like the
 * box's sides; its sample points join STK_PTS_BOUNDARY_FACE), and takes
 * p = 1..3, FP64 or FP32 blocks; clusters, the persistent launches, several
 * right-hand sides, the learned smoother and the autotuner are Cartesian
 * only.  r = 0 returns the context to the Cartesian mesh.  Call after
 * stk_set_discretisation.  Errors: STK_ERR_INVALID_ARG (not 2D, bad circle).
 */
int stk_set_levelset_circle(stk_ctx* ctx, double cx, double cy, double r);
/* Warps that share one element in the element kernel of cut-cell levels: 0
 * (default) picks by launch size (4 for launches of fewer than 8 elements per
 * SM with FP32 records or 32 with FP64 records, else 2), or 1, 2, 4 fixed.
 * Results agree to rounding (the warps' partial sums meet in a different
 * order).  Errors: STK_ERR_INVALID_ARG. */
int stk_set_element_warps(stk_ctx* ctx, int warps);
/* Unsteady cut-cell problem (eq. timedep2): density rho_phase > 0 per phase
 * of stk_set_phases (2 values, 1 for the disc) and delta > 0; delta = 0
 * returns to the steady problem (rho_phase unused).  Call after
 * stk_set_phases. */
int stk_set_phase_density(stk_ctx* ctx, const double* rho_phase, double delta);
/* Phase (1 or 2) of every point of a point set of a cut-cell mesh (volume and
 * boundary-face points: the phase of the piece they belong to; interface
 * points: 1, the inside).  Cut-cell point sets: STK_PTS_VOLUME (the pieces'
 * volume rules, pieces in order), STK_PTS_INTERIOR_FACE (empty),
 * STK_PTS_BOUNDARY_FACE (box-face parts, cells in order, per cell the high x
 * and high y faces then the low faces on the box's low sides), and
 * STK_PTS_INTERFACE (the circle's rule, cut cells in order, normals out of
 * the circle).  stk_assemble_rhs2 then takes f_vol [volume point][3] =
 * (f_1, f_2, fdiv), bdata [boundary point][2] = g, idata [interface
 * point][4] = (g_1, g_2, h_1, h_2) with g = u(1) - u(2) and
 * h = sigma(1) n - sigma(2) n. */
int stk_get_point_phases(stk_ctx* ctx, int kind, int* phase);

/* Bottom solve x = A_c^+ b on the last level (FP64). */
int stk_bottom_solve(stk_ctx* ctx, const double* b_dev, double* x_dev, void* stream);

/*
 * Convergence rate rho of eq. (rho) (Section 4): GMRES, not restarted, on the
 * left-preconditioned system V A x = V b with b = 0 from the initial guess
 * x0_dev (caller-owned device array [element][nb], FP64, not modified); V is
 * one cycle of the context's precision and shape from a zero guess.  Stops at
 * the first iteration n with ||V A x_n|| <= reduction ||V A x_0|| (the paper
 * uses 1e-8) or at maxit; *rho_out = (||V A x_n|| / ||V A x_0||)^(1/n),
 * *iters_out = n (may be NULL).  hist (host, maxit+1 entries, may be NULL):
 * the relative preconditioned residual per iteration.  hess (host,
 * (maxit+1) x maxit row-major, may be NULL): the Arnoldi matrix before the
 * Givens rotations; the eigenvalues of its leading n x n block estimate the
 * spectrum of V A (Section 4's spectral estimate).  An x0 with V A x0 = 0
 * gives rho = 0 after 0 iterations.  Errors: STK_ERR_NOT_SETUP,
 * STK_ERR_INVALID_ARG (reduction outside (0,1), maxit outside 1..100, NULL
 * x0_dev or rho_out), STK_ERR_TIMEOUT, STK_ERR_DIVERGED (a non-finite
 * residual).
 */
int stk_gmres_rho(stk_ctx* ctx, const double* x0_dev, double reduction, int maxit, double* rho_out,
                  int* iters_out, double* hist, double* hess, void* stream);

/*
 * Solve A x = b to ||b - A x||_2 <= rtol ||b||_2 by the outer iteration
 * x <- x + V(0, b - A x) (iterative refinement with the V-cycle of
 * stk_set_cycle's precision as preconditioner; residual in FP64).  x_dev
 * holds the initial guess.  *iters_out gets the iteration count, hist (may
 * be NULL, maxit+1 entries) the relative residual history.  Returns
 * STK_ERR_DIVERGED if the residual becomes non-finite or grows 1e6-fold.
 */
int stk_solve(stk_ctx* ctx, double* x_dev, const double* b_dev, double rtol, int maxit,
              int* iters_out, double* hist, void* stream);

/*
 * Allocation-free variant of stk_residual with the norm: r = b - A x on
 * level 0 in FP64 and ||r||_2^2 written to the caller's device scalar
 * *norm2_dev, enqueued on `stream` without synchronising.  The paper has no
 * counterpart; this entry point exists for callers that must not allocate
 * device memory while they run -- code under a fixed device-memory budget,
 * or a host thread that must not call cudaMalloc because it can block on or
 * serialise with work already running on the device.  The call allocates
 * nothing: its only scratch (the per-chunk partial sums of ||r||^2) is a
 * 128 KB file-scope device array that every GPU which loads the library holds
 * until the process exits.  Limits and caveats:
 *  - at most 33,554,432 unknowns on level 0 (16384 chunks of 2048);
 *    larger problems return STK_ERR_INVALID_ARG with a message;
 *  - the first call on a device looks up the array's device address (with
 *    that device made current) and caches it for the life of the process;
 *    make that first call before any stream capture; a cudaDeviceReset (or
 *    unloading the library) invalidates the cached address, so do not call
 *    this entry point again after one;
 *  - all calls share the array; each call writes every slot it reads, but
 *    calls that overlap on the GPU (e.g. on two streams) race on it;
 *  - on failure only the context's host-side error message is updated.
 */
int stk_residual_norm_static(stk_ctx* ctx, const double* x_dev, const double* b_dev, double* r_dev,
                             double* norm2_dev, void* stream);

/*
 * Several right-hand sides at once (up to 8): X and B are [nrhs][element][nb]
 * FP64 device arrays, X holding the initial guesses.  The V-cycle of
 * Algorithm 1 is applied to all right-hand sides together, so each element
 * record streamed from memory serves every right-hand side.  With
 * stk_set_solver method 1 or 2: flexible GMRES(restart) in FP64, run in
 * lockstep over the right-hand sides (one multi-RHS V-cycle and one FP64
 * multi-RHS matvec per step, dots and rotations per right-hand side, a
 * converged one drops out; restart capped at 256 / 8 = 32); *iters_out counts
 * Arnoldi steps.  With method 0: outer FP64 refinement X <- X + C with the
 * FP64 residual R = B - A X; inside, `inner` steps of C <- C + V(0, R - A C)
 * with the residual in the cycle's precision, one outer iteration as one CUDA
 * graph.  Stops when every ||B_q - A X_q|| <= rtol ||B_q|| or after maxit
 * iterations; hist (may be NULL) gets (maxit+1) x nrhs relative residuals.
 */
int stk_solve_multi(stk_ctx* ctx, double* X_dev, const double* B_dev, int nrhs, double rtol, int maxit, int inner,
                    int* iters_out, double* hist, void* stream);

/*
 * With eight right-hand sides (nrhs 5..8) and FP32 blocks, the element
 * products of stk_solve_multi are small dense GEMMs (each s x s coupling
 * sub-block times s x 8 neighbour values, the nb x nb block times nb x 8
 * values): on = 1 (default) computes them on the tensor cores (mma.sync
 * m16n8k8 TF32, each FP32 operand split into two TF32 parts, three products
 * accumulated in FP32, about FP32 accuracy); on = 0 on the FP32 CUDA cores.
 * Other precisions and four right-hand sides always use the CUDA cores.
 */
int stk_set_mrhs_tensor(stk_ctx* ctx, int on);

/*
 * The FP64 matvec of flexible GMRES (method 1) under an FP32, BF16 or FP16
 * cycle (no counterpart in the paper): the preconditioned vector z_j is the
 * cycle's FP32 output, so A z_j is formed from the level-0 FP32 records and
 * their FP32 remainders (A_hi + A_lo, ~48 bits) with exact FP32 products and
 * two-sum accumulation on the FP32 units, to about 2^-44 relative to
 * |A| |z_j| per entry, instead of on the FP64 units (64 times slower on this
 * GPU).  on = 1 (default) or 0 (FP64 records and arithmetic).  The outer
 * residual at each restart stays FP64.
 */
int stk_set_df_matvec(stk_ctx* ctx, int on);

/*
 * A batch of independent problems (no counterpart in the paper; a batching
 * layer over stk_solve / stk_solve_multi): solves ctx[i] x[i] = b[i] for
 * i < n, each context set up for its own problem (any mesh size, degree,
 * boundary conditions or precision; every context distinct).  A pool of
 * `threads` host threads (0: one per hardware thread, at most n) takes the
 * problems in order; each problem's whole outer iteration runs on its own
 * context's stream, so the kernels of different problems overlap on the GPU
 * (the coarse levels of one problem leave most SMs idle).  nrhs = 1 calls
 * stk_solve with the context's solver options; nrhs in 2..8 calls
 * stk_solve_multi with `inner` (x[i], b[i] then hold nrhs right-hand sides,
 * [nrhs][element][nb]).  The caller's `stream` is synchronised first.
 * iters_out and status_out (may be NULL, n entries) get each problem's
 * iteration count and status code; stk_last_error(ctx[i]) holds its message.
 * Returns STK_OK when every problem succeeded, else the first failing
 * problem's code.  Errors: STK_ERR_INVALID_ARG (null or repeated context,
 * n < 1, nrhs outside 1..8), STK_ERR_CUDA.
 */
/*
 * The same batch in ONE persistent launch (no counterpart in the paper): every
 * outer iteration of every problem runs inside a single cooperative kernel
 * of ctas_per_sm CTAs per SM.  The outer iteration is iterative refinement,
 * x <- x + V(0, b - A x), with the context's V-cycle shape on FP32 records
 * and the residual on the FP64 records; one iteration is a program of steps
 * (the cycle input, every colour step, residual, restriction, bottom solve
 * and prolongation of Algorithm 1, the update of x, the FP64 residual, its
 * norm, and the convergence test ||b - A x|| <= rtol ||b||), and step k of
 * all problems runs together -- a work list of (problem, step, element or
 * coarse element or chunk) units -- with a bounded grid barrier between
 * steps; each unit is one warp's (an element on the warp-per-element body of
 * the large launches, a coarse element, a bottom row, or a vector chunk).
 * A problem that converged (or diverged: non-finite, or 1e6 times its
 * initial residual) stops taking part; the launch ends when none is left or
 * after maxit iterations.  Every context must be set up with FP32 cycles,
 * distinct, on one device, for a degree with 4, 8, 9, 16 or 27 scalar modes
 * per element; their level work vectors are used, so no other call may use
 * them meanwhile.  x[i] (FP64 [element][nb], the initial guess, overwritten)
 * and b[i] are device arrays of the caller.  iters_out, status_out (n
 * entries) and hist (n x (maxit + 1): relative residual before the first and
 * after each iteration, zero beyond the last) may be NULL.  Every element of
 * every level runs on the warp-per-element body, so results agree with
 * stk_solve's (whose coarse levels take the one-CTA-per-element body) to
 * rounding, not bit for bit.  The workspace (work list,
 * partial sums) is allocated per call.  Errors: STK_ERR_INVALID_ARG,
 * STK_ERR_NOT_SETUP, STK_ERR_DIVERGED (status_out says which problem),
 * STK_ERR_TIMEOUT (a barrier wait reached its bound; messages in
 * stk_last_error(ctx[0])), STK_ERR_CUDA.
 */
int stk_solve_batch_persistent(stk_ctx* const* ctx, int n, double* const* x, const double* const* b, double rtol,
                               int maxit, int ctas_per_sm, int* iters_out, int* status_out, double* hist,
                               void* stream);
int stk_solve_batch(stk_ctx* const* ctx, int n, double* const* x, const double* const* b, int nrhs, double rtol,
                    int maxit, int inner, int threads, int* iters_out, int* status_out, void* stream);

/*
 * Learned element-local post-smoother (not in the paper; cycles in FP32 or
 * BF16 only).  After a V-cycle c = V(0, r) on the finest level, with
 * r_c = r - A c the cycle's own residual after its post-smoothing sweeps
 * (FP32, the cycle's records), each element's r_c,i and those of its 2d face
 * neighbours, divided by ||r_c,i||, go through a two-layer perceptron
 * (in = (2d+1) nb, tanh hidden layer of `hidden` units, out = nb) whose
 * output times ||r_c,i|| is a correction delta_i.
 * Acceptance (kept only where its measured contraction beats plain block
 * Gauss-Seidel): stk_solve with outer method 0 (iterative refinement) runs
 * its first two iterations with plain cycles and measures their contraction
 * kappa = (||r_2|| / ||r_0||)^(1/2); every later iteration applies
 * x <- x + c + delta and keeps delta only if the new FP64 outer residual
 * (computed anyway) satisfies ||r_new|| < kappa ||r_old||; otherwise delta is
 * subtracted again (x + c, the plain cycle's result, with its residual
 * recomputed), and after two consecutive rejections the correction is
 * switched off for the rest of that solve.  The plain smoother is thus both
 * the fallback and the yardstick.  stk_solve with a Krylov outer method and
 * the correction enabled returns STK_ERR_INVALID_ARG (the rule needs the
 * outer residual of every cycle).
 *  stk_learn_setup     allocate and initialise the weights (deterministic in seed);
 *  stk_learn_generate  training states from the plain V-cycle: for nseeds smooth
 *                      random solutions x* (seeded), b = A x*, `cycles` V-cycles
 *                      from zero, storing r = b - A x and e = x* - x after each;
 *  stk_learn_objective 0 (default): Adam minimises ||r - A delta(r)||^2 / ||r||^2;
 *                      1: the supervised error target, the mean over elements
 *                      of ||delta_i / ||r_i|| - e_i / ||r_i||||^2 (MSE of the
 *                      per-element normalised error);
 *  stk_learn_train     Adam on the chosen objective over the stored states in
 *                      random order (`epochs` passes; `batch` is unused, one
 *                      state per step); *loss_out = mean loss of the last pass;
 *  stk_learn_enable    apply (1) or drop (0) the correction in stk_solve;
 *  stk_learn_stats     outer iterations whose correction was kept / undone
 *                      since stk_learn_enable;
 *  stk_learn_history   per outer iteration of the last stk_solve: decision[k]
 *                      = -1 plain cycle (kappa measurement, or switched off),
 *                      1 kept, 0 undone, and ratio[k] = ||r_new|| /
 *                      (kappa ||r_old||) of the judged iterations (0 for
 *                      plain ones); *count = iterations (at most max entries
 *                      are written); *kappa_out = kappa;
 *  stk_learn_weights   copy the weights to (direction 0) or from (1) a host array.
 */
int stk_learn_setup(stk_ctx* ctx, int hidden, uint64_t seed);
int stk_learn_generate(stk_ctx* ctx, int nseeds, int cycles, uint64_t seed);
int stk_learn_train(stk_ctx* ctx, int epochs, int batch, double lr, uint64_t seed, double* loss_out);
int stk_learn_enable(stk_ctx* ctx, int on);
int stk_learn_stats(stk_ctx* ctx, int64_t* accepted, int64_t* rejected);
int stk_learn_weights(stk_ctx* ctx, float* host, int64_t count, int direction);
/* The smooth random field of the training data for hash seed `seed` (sample k
 * of stk_learn_generate(..., seed0) uses seed0 + 7919 k) into the caller's
 * FP64 device vector x [element][nb]: per variable a sum of four seeded
 * sines of the element centre (mode 0) plus 1e-3 seeded noise on the higher
 * modes.  For evaluation right-hand sides b = A x from seeds the training did
 * not use.  Needs stk_learn_setup. */
int stk_learn_field(stk_ctx* ctx, uint64_t seed, double* x_dev, void* stream);
int stk_learn_objective(stk_ctx* ctx, int objective);
int stk_learn_history(stk_ctx* ctx, int* decision, double* ratio, int max, int* count, double* kappa_out);
/* Sizes: input width (2d+1) nb, hidden width, output nb, number of weights
 * (W1 [in][hidden], b1, W2 [hidden][nb], b2, packed in that order), number
 * of stored residual states. */
int stk_learn_sizes(stk_ctx* ctx, int* in, int* hidden, int* out, int64_t* nparam, int64_t* states);
/* Features of a finest-level FP32 residual r_dev [element][nb] and the MLP
 * output y_dev [element][nb] (before the ||r_i|| scaling), nrm_dev [element]. */
int stk_learn_infer(stk_ctx* ctx, const float* r_dev, float* y_dev, float* nrm_dev);
/* Host copies of a stored residual state r (stk_learn_state) and of the error
 * e = x* - x stored with it (stk_learn_error_state), and the training loss of
 * the current objective and its gradient (host, packed like the weights) on
 * that state, without updating the weights. */
int stk_learn_state(stk_ctx* ctx, int64_t state, float* r);
int stk_learn_error_state(stk_ctx* ctx, int64_t state, float* e);
int stk_learn_grad(stk_ctx* ctx, int64_t state, float* grad, double* loss_out);

/*
 * Outer iteration of stk_solve: method 0 = iterative refinement
 * x <- x + V(0, b - A x) (default); method 1 = flexible GMRES(restart) in
 * FP64 with one V-cycle (of the stk_set_cycle precision, from a zero guess)
 * as the right preconditioner -- Section 3 uses the V-cycle as a GMRES
 * preconditioner; the flexible form keeps the FP64 residual exact when the
 * cycle runs in FP32/BF16.  method 2 = the same flexible GMRES with the
 * Krylov matvec on FP32 blocks and vectors (also when the cycle runs in BF16),
 * trusted for a 1e-5 reduction per restart cycle, inside FP64 refinement:
 * each restart recomputes the residual in FP64.  With an FP64 cycle method 2
 * equals method 1.  restart in 1..100.
 */
int stk_set_solver(stk_ctx* ctx, int method, int restart);

/*
 * Kernel tuning for the element kernel (colour steps and residuals):
 * variant 0 = one CTA per element with direct 16-byte loads of the element
 * records; variant 1 = the records streamed into a shared-memory ring of
 * `stages` buffers by 1-D bulk copies (cp.async.bulk, mbarrier completion);
 * variant 2 (default for FP64 and FP32 blocks) = one warp per element, no
 * block-wide barriers;
 * variant 3 = one or two warps per element whose records, scales and
 * gathered neighbour values are copied into their shared memory by cp.async,
 * the next element's coupling records while they compute this element's
 * dense product (the default for BF16 and FP16
 * blocks, s and nb multiples of 4, at most 32 neighbour offsets; other
 * shapes and precisions run variant 2; the same products as variant 2, each
 * coupling row summed as two halves of its columns).
 * The variant and `ctas_per_sm` (the grid of variants 1 and 2, CTAs per SM;
 * for variant 3 the warps per element: 1, 4, or 2 (the default: four on
 * launches of at most six elements per SM)) apply to the
 * blocks stored in `precision` only.  Zero for ctas_per_sm and stages selects the
 * built-in shape for the record size.
 * Shapes whose ring does not fit in shared memory fall back to variant 0.
 * If a bulk copy never completes, the kernel's bounded wait (about one
 * second) expires and stk_solve returns STK_ERR_TIMEOUT.
 */
int stk_set_tuning(stk_ctx* ctx, int variant, int precision, int ctas_per_sm, int stages);

/*
 * Launch overlap for the element kernels (not in the paper): on = 1 (the
 * default) launches the colour steps and residuals of the warp (variant 2),
 * staged (variant 3), one-CTA-per-element (coarse levels) and cut-cell
 * kernels with programmatic stream serialisation, so that their CTAs start
 * while the previous kernel on the stream (a colour step, a transfer or the
 * bottom solve, each of which lets its dependents start at once) is still
 * running.  The staged, one-CTA-per-element and cut-cell kernels first
 * request what no launch writes (their first element's records, the dense
 * blocks, neighbour indices); every kernel then waits for the previous one
 * to complete and its writes to be visible before it reads or writes any
 * vector.  Results are unchanged bit for bit; on = 0 launches them plainly.
 * Errors: STK_ERR_INVALID_ARG unless on is 0 or 1.
 */
int stk_set_launch_overlap(stk_ctx* ctx, int on);

/*
 * Element-kernel launches over at most max_positions elements (the colour
 * steps and residuals of coarse levels) use one CTA of 256 threads per
 * element instead of the configured variant: with few elements per launch
 * the time is one element's load latency, which a whole CTA shortens by
 * issuing all of the element's record loads at once.  Same arithmetic per
 * row (FP32/FP64 sums in a different association order).  The same limit
 * sends eight-right-hand-side tensor-core launches to their four-warps-per-
 * element kernel.  0 disables it; default 1024.  Errors: STK_ERR_INVALID_ARG
 * for a negative value.
 */
int stk_set_wide_launch(stk_ctx* ctx, int max_positions);

/*
 * Autotuner for the element-kernel launches (no counterpart in the paper):
 * on this context's own finest-level records it times one colour step for
 * the warp-per-element kernel at 2, 3, 4, 6 and 8 CTAs per SM, for the
 * one-CTA-per-element kernel with direct loads and, for 16-bit blocks, for
 * the staged kernel (variant 3) with one and two warps per element, in the
 * cycle's precision and
 * in FP64 (the outer residual), and keeps the fastest shapes; then it times
 * both that choice and the one-CTA-per-element latency kernel on every
 * smoothing level and sets the stk_set_wide_launch threshold with the least
 * total time.  Each timing replays a CUDA graph of repeated launches on the
 * library's own stream, so host launch overhead does not mask the kernels.
 * Call after stk_setup, outside any stream capture; it runs colour steps on
 * the library's own work vectors (zeroed before and after) and synchronises
 * `stream`.  The variant and the CTAs per SM are kept per storage precision
 * (the FP64 outer residual may take another kernel than the cycle); under a
 * low-precision cycle it also times the two FGMRES matvecs (stk_set_df_matvec)
 * over level 0 and keeps the faster.  choice (may be NULL, 6 ints) receives
 * {variant and CTAs per SM (variant 3: warps per element) in the cycle
 * precision, variant and CTAs per SM in
 * FP64, latency-kernel limit, FP32-unit matvec on/off};
 * best_ms (may be NULL, 2 doubles) the fastest finest-level colour step in
 * the cycle precision and in FP64.  Results are unchanged up to the
 * association order of sums.  Errors: STK_ERR_NOT_SETUP, STK_ERR_CUDA.
 */
int stk_autotune(stk_ctx* ctx, int* choice, double* best_ms, void* stream);

/* Number of kernel launches the library enqueued since the context was
 * created (all of them are this library's own kernels). */
int stk_launch_count(stk_ctx* ctx, int64_t* count);

/*
 * Measured FP64 FMA rate of the context's device (not a step of the method;
 * it is the denominator of the FP64 element kernels' roofline, whose
 * arithmetic intensity of 0.25 flop/B can be bound by the FP64 pipe rather
 * than by HBM).  A project kernel runs eight independent FMA chains per
 * thread on 8 CTAs of 256 threads per SM, 2^16 FMAs per chain; *tflops gets
 * the best of three timed launches (CUDA events on `stream`, after one
 * warm-up), in TFLOP/s counting 2 flops per FMA.  Needs stk_setup.
 */
int stk_fp64_fma_rate(stk_ctx* ctx, double* tflops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* STOKES_MG_H */
