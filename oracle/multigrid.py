"""Block Gauss-Seidel V-cycle for the LDG Stokes system (oracle).

Section 3 (Multigrid design):
  * Block Gauss-Seidel: blocks are all velocity and pressure unknowns of one
    element; x_i <- A_ii^{-1} (b_i - sum_{j != i} A_ij x_j).  The sweep is
    multi-coloured (colour sum_k (i_k mod 2) 2^k, colours in ascending order,
    every element of one colour updated from the same x); a lexicographic
    (element-order) sweep is kept as the second reference.
  * Algorithm 1: V(E_h, x_h, b_h) with nu1 pre- and nu2 post-smoothing sweeps,
    r_2h = (I_2h^h)^T (b_h - A_h x_h), coarse guess 0, x_h += I_2h^h x_2h.
  * Section 6's alternatives to the V-cycle: W-cycles (gamma coarse visits
    per level) and variable V-cycles (smoothing counts growing per level);
    the Concluding Remarks' element clustering (blocks of 2^d elements on the
    finest level) as a smoother option.
  * Bottom solver (Section 3 footnote on the trivial kernel): symmetric
    eigendecomposition of the coarsest operator with near-zero eigenvalues
    snapped to zero (least-squares solution).
  * V-cycle-preconditioned GMRES (left preconditioning, not restarted) and the
    convergence rate rho of eq. (rho).

Readings: post-smoothing visits the colours in the same ascending order; the
snap threshold is |lambda| <= 1e-10 max|lambda|; the A_ii^{-1} applied by the
smoother is the explicit inverse (numpy.linalg.inv); the outer iteration is
x <- x + V(0, b - A x) until ||b - A x||_2 <= rtol ||b||_2.

Low-precision storage (not in the paper; emulated here as the library stores
it): every block of the smoother -- A_ii^{-1}, A_ii and the couplings -- is
rounded once from FP64, and a cycle with rounded blocks also forms its
in-cycle residual b - A x from those rounded blocks (the outer residual stays
FP64).  precondition() keeps vectors and sums in FP64; precondition_fp32()
runs the same cycle on float32 vectors with float32 products and sums (the
library's FP32 cycle: FP32 vectors on every level, the injection rounded to
FP32, the bottom pseudo-inverse applied in FP64 to the float32 right-hand side
and rounded back).
"""
import numpy as np
import scipy.sparse as sp

from .hierarchy import build_hierarchy, diag_blocks

SNAP_THETA = 1e-10


def round_fp32(a):
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_fp16_scaled(a, axis):
    """Round to IEEE binary16 (round to nearest even) with one power-of-two
    scale per group of entries, a group being the entries that share all
    indices except those of `axis`: with 2^(e-1) <= max|a| < 2^e over the
    group, the entries are multiplied by 2^(15-e) (largest magnitude in
    [2^14, 2^15)), rounded, and multiplied back.  An all-zero group stays zero."""
    a = np.asarray(a, dtype=np.float64)
    mx = np.abs(a).max(axis=axis, keepdims=True)
    _, e = np.frexp(mx)
    e = np.where(mx > 0, e, 0).astype(np.float64)
    up = np.exp2(15.0 - e)
    return (a * up).astype(np.float16).astype(np.float64) / up


def round_fp16_subblocks(A, s):
    """round_fp16_scaled on a sparse matrix whose groups are its s x s
    sub-blocks (row block i, column block j), as scipy CSR."""
    coo = sp.coo_matrix(A)
    nbc = A.shape[1] // s
    key = (coo.row // s).astype(np.int64) * nbc + coo.col // s
    uniq, inv = np.unique(key, return_inverse=True)
    mx = np.zeros(len(uniq))
    np.maximum.at(mx, inv, np.abs(coo.data))
    _, e = np.frexp(mx)
    e = np.where(mx > 0, e, 0).astype(np.float64)
    up = np.exp2(15.0 - e)[inv]
    data = (coo.data * up).astype(np.float16).astype(np.float64) / up
    return sp.csr_matrix((data, (coo.row, coo.col)), shape=A.shape)


def round_bf16(a):
    """Round to bfloat16 (round to nearest even from the fp32 value)."""
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


class SmootherLevel:
    """Smoother data of one level: A_ii, A_ii^{-1}, and the off-block-diagonal
    part of A restricted to the rows of each colour."""

    def __init__(self, lev, storage=None, two_colours=False):
        self.lev = lev
        self.nb = lev.nb
        self.ne = lev.ne
        A = lev.A
        self.diag = diag_blocks(A, self.ne, self.nb)
        self.inv = np.linalg.inv(self.diag)
        coo = A.tocoo()
        off = (coo.row // self.nb) != (coo.col // self.nb)
        self.Aoff = sp.csr_matrix((coo.data[off], (coo.row[off], coo.col[off])), shape=A.shape)
        if storage == "fp32":
            self.inv = round_fp32(self.inv)
            self.Aoff.data = round_fp32(self.Aoff.data)
            self.diag = round_fp32(self.diag)
        elif storage == "bf16":
            self.inv = round_bf16(self.inv)
            self.Aoff.data = round_bf16(self.Aoff.data)
            self.diag = round_bf16(self.diag)
        elif storage == "fp16":
            # one scale per row of A_ii^{-1} and of A_ii, one per s x s coupling sub-block
            self.inv = round_fp16_scaled(self.inv, axis=2)
            self.diag = round_fp16_scaled(self.diag, axis=2)
            self.Aoff = round_fp16_subblocks(self.Aoff, lev.s)
        self.colour = lev.mesh.colour_two() if two_colours else lev.mesh.colour()
        self.ncol = int(self.colour.max()) + 1
        self.elems = [np.nonzero(self.colour == c)[0] for c in range(self.ncol)]
        self.rows = [(e[:, None] * self.nb + np.arange(self.nb)[None, :]).ravel() for e in self.elems]
        self.Aoff_rows = [self.Aoff[r, :].tocsr() for r in self.rows]

    def f32(self):
        """float32 copies of the blocks (for a float32 cycle)."""
        if not hasattr(self, "_f32"):
            self._f32 = (self.inv.astype(np.float32), self.diag.astype(np.float32),
                         [m.astype(np.float32) for m in self.Aoff_rows], self.Aoff.astype(np.float32))
        return self._f32

    def colour_step(self, x, b, c):
        """Update every element of colour c from the current x (one data-parallel step).
        float32 vectors take float32 products and sums."""
        r = self.rows[c]
        if x.dtype == np.float32:
            inv, _, rows, _ = self.f32()
            g = (b[r] - rows[c] @ x).reshape(-1, self.nb)
            x[r] = np.einsum("eij,ej->ei", inv[self.elems[c]], g).ravel()
            return
        g = (b[r] - self.Aoff_rows[c] @ x).reshape(-1, self.nb)
        x[r] = np.einsum("eij,ej->ei", self.inv[self.elems[c]], g).ravel()

    def sweep(self, x, b):
        for c in range(self.ncol):
            self.colour_step(x, b, c)

    def sweep_lexicographic(self, x, b):
        """Element-order block Gauss-Seidel (no colours)."""
        nb = self.nb
        A = self.Aoff
        for i in range(self.ne):
            sl = slice(i * nb, (i + 1) * nb)
            g = b[sl] - A[sl, :] @ x
            x[sl] = self.inv[i] @ g


def cluster_layout(mesh):
    """Clusters of 2^d elements (the 2 x 2 (x 2) children of one cell of the
    mesh with halved n): the cluster index of every element and its child
    position ch = sum_k (i_k mod 2) 2^k, and the cluster grid."""
    idx = mesh.idx
    nc = [n // 2 for n in mesh.n]
    cstride = [int(np.prod(nc[:k])) for k in range(mesh.d)]
    cid = ((idx // 2) * np.asarray(cstride)).sum(axis=1)
    child = ((idx % 2) * (2 ** np.arange(mesh.d))).sum(axis=1)
    cidx = np.stack([(np.arange(int(np.prod(nc))) // cstride[k]) % nc[k] for k in range(mesh.d)], axis=1)
    return cid, child, nc, cidx


def clusters_apply(mesh, gamma):
    """Element clustering (Concluding Remarks: larger smoother blocks for
    p = 1) is used on a level when every axis has an even element count and
    every periodic axis an even cluster count (so that the cluster colouring
    closes around the wrap), on single-phase problems."""
    if mesh.chi is not None:
        return False
    for k in range(mesh.d):
        if mesh.n[k] % 2:
            return False
        if mesh.periodic(k) and (mesh.n[k] // 2) % 2:
            return False
    return True


class ClusterSmootherLevel:
    """Block Gauss-Seidel over clusters of 2^d elements: each block is every
    unknown of the 2^d children of one coarse cell, x_C <- A_CC^{-1}(b_C -
    sum_{D != C} A_CD x_D); clusters coloured like elements one level down
    (checkerboard of the cluster index for the standard form, whose clusters
    couple across faces only; 2^d parity colours otherwise), colours in
    ascending order."""

    def __init__(self, lev):
        self.lev = lev
        mesh = lev.mesh
        nb = lev.nb
        cid, child, nc, cidx = cluster_layout(mesh)
        self.ncl = int(np.prod(nc))
        self.rows = []
        for C in range(self.ncl):
            els = np.nonzero(cid == C)[0]
            els = els[np.argsort(child[els])]
            self.rows.append((els[:, None] * nb + np.arange(nb)[None, :]).ravel())
        A = lev.A.tocsr()
        self.blocks = [A[r][:, r].toarray() for r in self.rows]
        self.inv = [np.linalg.inv(B) for B in self.blocks]
        self.Arows = [A[r] for r in self.rows]
        if lev.standard_form:
            self.colour = cidx.sum(axis=1) % 2
        else:
            self.colour = (cidx % 2 * (2 ** np.arange(mesh.d))).sum(axis=1)
        self.ncol = int(self.colour.max()) + 1

    def colour_step(self, x, b, c):
        """Update every cluster of colour c from the current x."""
        for C in np.nonzero(self.colour == c)[0]:
            r = self.rows[C]
            g = b[r] - self.Arows[C] @ x + self.blocks[C] @ x[r]
            x[r] = self.inv[C] @ g

    def sweep(self, x, b):
        for c in range(self.ncol):
            self.colour_step(x, b, c)

    def sweep_lexicographic(self, x, b):
        for C in range(self.ncl):
            r = self.rows[C]
            x[r] = self.inv[C] @ (b[r] - self.Arows[C] @ x + self.blocks[C] @ x[r])


def bottom_pseudo_inverse(A, theta=SNAP_THETA):
    """Least-squares inverse of the coarsest operator: eigendecomposition with
    |lambda| <= theta max|lambda| snapped to zero.  Returns (pinv, n_snapped)."""
    Ad = A.toarray()
    Ad = 0.5 * (Ad + Ad.T)
    lam, V = np.linalg.eigh(Ad)
    keep = np.abs(lam) > theta * np.abs(lam).max()
    inv = np.where(keep, 1.0 / np.where(keep, lam, 1.0), 0.0)
    return (V * inv[None, :]) @ V.T, int((~keep).sum())


class Multigrid:
    """The V-cycle hierarchy of a problem (oracle)."""

    def __init__(self, prob, storage=None, levels=None, injections=None, max_levels=None, shape=(1, 1, 64),
                 two_colours=False, clusters=False):
        self.prob = prob
        # cycle shape (Section 6): coarse visits per level (1 V, 2 W), growth
        # of the smoothing counts per coarser level, cap on the counts
        self.gamma, self.growth, self.max_sweeps = shape
        if levels is None:
            levels, injections = build_hierarchy(prob, max_levels=max_levels)
        self.levels = levels
        self.I = injections
        self.storage = storage
        # two_colours: the checkerboard instead of the 2^d parity colours
        # (valid for face-coupled operators only: gamma = 0, single phase)
        self.sm = [SmootherLevel(l, storage, two_colours) for l in levels[:-1]]
        # clusters: the finest level smooths 2^d-element clusters (FP64 blocks)
        self.clusters = False
        if clusters and storage is None and clusters_apply(levels[0].mesh, prob.gamma):
            levels[0].standard_form = prob.gamma == 0
            self.sm[0] = ClusterSmootherLevel(levels[0])
            self.clusters = True
        self.bottom, self.kernel_dim_bottom = bottom_pseudo_inverse(levels[-1].A)
        self.nu1, self.nu2 = prob.nu1, prob.nu2

    @property
    def A(self):
        return self.levels[0].A

    def scale_rhs(self, b):
        """b~ = D b for the sqrt(mu)-scaled system (identity without scaling)."""
        D = self.levels[0].D
        return b if D is None else D * b

    def unscale(self, x):
        """x = D x~ (identity without scaling)."""
        D = self.levels[0].D
        return x if D is None else D * x

    def bottom_solve(self, b, refine=3):
        """Least-squares solution A_c^+ b of the bottom level (Section 3
        footnote).  The eigen pseudo-inverse is applied and then refined in
        FP64, x <- x + A_c^+ (b - A_c x): the eigendecomposition alone leaves a
        relative error of about 1e-12 on these operators, the refined result is
        the least-squares solution to rounding level."""
        A = self.levels[-1].A
        x = self.bottom @ b
        for _ in range(refine):
            x = x + self.bottom @ (b - A @ x)
        return x

    def residual(self, l, x, b):
        return b - self.levels[l].A @ x

    def cycle_residual(self, l, x, b):
        """Residual inside the V-cycle: from the smoother's stored blocks
        (rounded ones for a low-precision cycle; = residual() in FP64)."""
        if x.dtype == np.float32:
            sm = self.sm[l]
            _, diag, _, Aoff = sm.f32()
            y = np.einsum("eij,ej->ei", diag, x.reshape(-1, sm.nb)).ravel()
            return b - (y + Aoff @ x)
        if self.storage is None:
            return self.residual(l, x, b)
        sm = self.sm[l]
        y = np.einsum("eij,ej->ei", sm.diag, x.reshape(-1, sm.nb)).ravel()
        return b - (y + sm.Aoff @ x)

    def _I32(self, l):
        if not hasattr(self, "_i32"):
            self._i32 = [m.astype(np.float32) for m in self.I]
        return self._i32[l]

    def restrict(self, l, r):
        """r_2h = (I_2h^h)^T r_h, the coarse right-hand side of Algorithm 1."""
        if r.dtype == np.float32:
            return self._I32(l).T @ r
        return self.I[l].T @ r

    def prolong(self, l, xc):
        """I_2h^h x_2h (injection)."""
        if xc.dtype == np.float32:
            return self._I32(l) @ xc
        return self.I[l] @ xc

    def sweeps(self, nu, l):
        """Smoothing sweeps of one phase on level l.  Section 6 names the
        variable V-cycle, whose smoothing counts change from level to level;
        here they grow geometrically, nu * growth^l, up to max(nu, cap).
        growth = 1 gives Algorithm 1's fixed counts."""
        return min(nu * self.growth ** l, max(nu, self.max_sweeps))

    def vcycle(self, x, b, l=0, nu1=None, nu2=None, lexicographic=False):
        """Algorithm 1: returns x after one V-cycle (x is updated in place).
        With gamma > 1 the coarse problem of every level is visited gamma
        times (the W-cycle for gamma = 2, Section 6), the first visit from a
        zero guess and each later one from the previous result; the coarsest
        level is solved exactly, so it is visited once."""
        nu1 = self.nu1 if nu1 is None else nu1
        nu2 = self.nu2 if nu2 is None else nu2
        if l == len(self.levels) - 1:
            if x.dtype == np.float32:
                x[:] = (self.bottom @ b.astype(np.float64)).astype(np.float32)
            else:
                x[:] = self.bottom_solve(b)
            return x
        sm = self.sm[l]
        for _ in range(self.sweeps(nu1, l)):
            (sm.sweep_lexicographic if lexicographic else sm.sweep)(x, b)
        r2 = self.restrict(l, self.cycle_residual(l, x, b))
        x2 = np.zeros_like(r2)
        visits = 1 if l + 1 == len(self.levels) - 1 else self.gamma
        for _ in range(visits):
            self.vcycle(x2, r2, l + 1, nu1, nu2, lexicographic)
        x += self.prolong(l, x2)
        for _ in range(self.sweeps(nu2, l)):
            (sm.sweep_lexicographic if lexicographic else sm.sweep)(x, b)
        return x

    def precondition(self, r, **kw):
        """The linear operator V: one V-cycle from a zero initial guess."""
        c = np.zeros_like(r)
        return self.vcycle(c, r, **kw)

    def precondition_fp32(self, r, **kw):
        """V on float32 vectors with float32 products and sums (the library's
        FP32 cycle): r rounded to float32, the result returned in FP64."""
        r32 = r.astype(np.float32)
        c = np.zeros_like(r32)
        return self.vcycle(c, r32, **kw).astype(np.float64)

    def solve(self, b, x0=None, rtol=1e-10, maxit=100, **kw):
        """Outer iteration x <- x + V(0, b - A x) (iterative refinement)."""
        x = np.zeros_like(b) if x0 is None else x0.copy()
        nb_ = np.linalg.norm(b)
        hist = []
        for it in range(maxit + 1):
            r = b - self.A @ x
            rel = np.linalg.norm(r) / nb_
            hist.append(rel)
            if rel <= rtol or it == maxit:
                break
            x += self.precondition(r, **kw)
        return x, hist

    def fgmres(self, b, x0=None, rtol=1e-10, maxit=200, restart=30, **kw):
        """Flexible right-preconditioned GMRES with the V-cycle as the
        preconditioner (Section 3 uses V as a GMRES preconditioner; the flexible
        form also admits a preconditioner that changes between iterations).
        Returns (x, history of ||b - A x|| / ||b|| per iteration)."""
        A = self.A
        x = np.zeros_like(b) if x0 is None else x0.copy()
        bn = np.linalg.norm(b)
        r = b - A @ x
        hist = [np.linalg.norm(r) / bn]
        it = 0
        while hist[-1] > rtol and it < maxit:
            beta = np.linalg.norm(r)
            V = [r / beta]
            Z = []
            H = np.zeros((restart + 1, restart))
            g = np.zeros(restart + 1)
            g[0] = beta
            cs, sn = np.zeros(restart), np.zeros(restart)
            k = 0
            for j in range(restart):
                z = self.precondition(V[j], **kw)
                Z.append(z)
                w = A @ z
                for i in range(j + 1):
                    H[i, j] = np.dot(V[i], w)
                    w = w - H[i, j] * V[i]
                H[j + 1, j] = np.linalg.norm(w)
                V.append(w / H[j + 1, j] if H[j + 1, j] > 0 else w)
                for i in range(j):
                    t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                    H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                    H[i, j] = t
                den = np.hypot(H[j, j], H[j + 1, j])
                cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
                H[j, j] = den
                H[j + 1, j] = 0.0
                g[j + 1] = -sn[j] * g[j]
                g[j] = cs[j] * g[j]
                k = j + 1
                it += 1
                hist.append(abs(g[j + 1]) / bn)
                if hist[-1] <= rtol or it >= maxit:
                    break
            y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
            x = x + np.array(Z[:k]).T @ y
            r = b - A @ x
            hist[-1] = np.linalg.norm(r) / bn
        return x, hist

    def gmres_rho(self, x0, reduction=1e-8, maxit=200, details=False, **kw):
        """eq. (rho): average reduction per iteration of left-preconditioned
        GMRES on V A x = V b with b = 0 from x0; returns (rho, iterations),
        with details=True also the relative preconditioned residual per
        iteration and the Arnoldi matrix before the Givens rotations (its
        leading n x n block's eigenvalues estimate the spectrum of V A, the
        estimate Section 4 uses)."""
        A = self.A

        def op(v):
            return self.precondition(A @ v, **kw)

        r0 = -op(x0)
        beta = np.linalg.norm(r0)
        Q = [r0 / beta]
        H = np.zeros((maxit + 1, maxit))
        cs, sn = np.zeros(maxit), np.zeros(maxit)
        g = np.zeros(maxit + 1)
        g[0] = beta
        n = 0
        Hraw = np.zeros_like(H)
        hist = [1.0]
        for j in range(maxit):
            w = op(Q[j])
            for i in range(j + 1):
                H[i, j] = np.dot(Q[i], w)
                w = w - H[i, j] * Q[i]
            H[j + 1, j] = np.linalg.norm(w)
            Hraw[: j + 2, j] = H[: j + 2, j]
            Q.append(w / H[j + 1, j] if H[j + 1, j] > 0 else w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            n = j + 1
            hist.append(abs(g[n]) / beta)
            if abs(g[j + 1]) <= reduction * beta:
                break
        rho = float(np.exp(np.log(abs(g[n]) / beta) / n))
        if details:
            return rho, n, np.array(hist), Hraw
        return rho, n
