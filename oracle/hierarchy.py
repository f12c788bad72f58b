"""Operator coarsening and the Stokes operator on every level (oracle).

Appendix B (operator coarsening geometric multigrid methods):
  * Algorithm 2 (steady): M_2h = I^T M_h I, M_mu,2h = I^T M_mu,h I,
    G_2h = M_2h^{-1} I^T M_h G_h I, E~_2h = 1/2 I^T E~_h I, E_2h = 2 I^T E_h I.
  * Algorithm 3 (unsteady): additionally M_rho,2h = I^T M_rho,h I,
    E_mu,2h = 2 I^T E_mu,h I, E_rho,2h = 1/2 I^T E_rho,h I, combined per
    element-pair block by eq. (Etimedep).
  * The Stokes operator of eq. (blockform) / (timedep2) with the viscous
    blocks of eq. (viscousop):
        A_ij = delta_ij (sum_k G_k^T M_mu G_k + E~ [+ M_rho/delta]) + gamma G_j^T M_mu G_i,
        upper right M Gcal_i, lower left Gcal_i^T M, Gcal_i = -M^{-1} G_i^T M,
        lower right -E.

The interpolation I_2h^h is injection (Section 3, "Interpolation operator"):
(I u)|_{E_f} = u|_{E_c}.

Readings: the hierarchy halves every axis while all n_k are even and at least
4; the last level (some n_k odd or equal to 2) is the bottom level.  On the
finest level of an unsteady problem E is assembled from eq. (taupgeneral);
eq. (Etimedep) is applied from the first coarse level down; a block pair with
||E_mu||_F + ||E_rho||_F = 0 gives a zero block.
"""
import numpy as np
import scipy.sparse as sp

from . import basis
from .ldg import Mesh, fine_operators


def injection(mesh_f, mesh_c, p):
    """Scalar injection matrix I (fine unknowns x coarse unknowns)."""
    d = mesh_f.d
    s = (p + 1) ** d
    P1 = [basis.child_1d(p, 0), basis.child_1d(p, 1)]
    child = mesh_f.idx % 2
    parent_idx = mesh_f.idx // 2
    parent = (parent_idx * np.asarray(mesh_c.stride)).sum(axis=1)
    rows, cols, vals = [], [], []
    a = np.arange(s)
    cache = {}
    for f in range(mesh_f.ne):
        key = tuple(child[f])
        if key not in cache:
            cache[key] = basis.kron_axes([P1[c] for c in key])
        P = cache[key]
        rows.append(np.repeat(f * s + a, s))
        cols.append(np.tile(parent[f] * s + a, s))
        vals.append(P.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(mesh_f.ne * s, mesh_c.ne * s))


def diag_blocks(Mat, ne, s):
    """The ne diagonal s x s blocks of a sparse matrix, as an array [ne, s, s]."""
    coo = Mat.tocoo()
    keep = (coo.row // s) == (coo.col // s)
    blocks = np.zeros((ne, s, s))
    np.add.at(blocks, (coo.row[keep] // s, coo.row[keep] % s, coo.col[keep] % s), coo.data[keep])
    return blocks


def blockdiag_inverse(Mat, ne, s):
    """Inverse of a block-diagonal matrix with s x s element blocks."""
    from .ldg import blocks_to_csr
    inv = np.linalg.inv(diag_blocks(Mat, ne, s))
    e = np.arange(ne)
    return blocks_to_csr(ne, s, e, e, inv)


def combine_pressure_penalty(Emu, Erho, ne, s):
    """eq. (Etimedep): per element-pair block (i, j),
    E_ij = (|E_rho,ij| / (|E_mu,ij| + |E_rho,ij|))^2 E_mu,ij
         + (|E_mu,ij| / (|E_mu,ij| + |E_rho,ij|))^2 E_rho,ij   (Frobenius norms)."""
    B = sp.kron(sp.identity(ne), np.ones((s, 1)), format="csr")  # (ne s) x ne
    Fmu = (B.T @ Emu.multiply(Emu) @ B).tocsr()
    Frho = (B.T @ Erho.multiply(Erho) @ B).tocsr()
    U = (abs(Fmu) + abs(Frho)).tocoo()
    fm = np.sqrt(np.asarray(Fmu[U.row, U.col]).ravel())
    fr = np.sqrt(np.asarray(Frho[U.row, U.col]).ravel())
    tot = fm + fr
    with np.errstate(invalid="ignore", divide="ignore"):
        wmu = np.where(tot > 0, (fr / tot) ** 2, 0.0)
        wrho = np.where(tot > 0, (fm / tot) ** 2, 0.0)
    Wmu = sp.csr_matrix((wmu, (U.row, U.col)), shape=(ne, ne))
    Wrho = sp.csr_matrix((wrho, (U.row, U.col)), shape=(ne, ne))
    Wmu_full = B @ Wmu @ B.T
    Wrho_full = B @ Wrho @ B.T
    return (Emu.multiply(Wmu_full) + Erho.multiply(Wrho_full)).tocsr()


def coarsen(ops, I, mesh_c, unsteady):
    """Algorithm 2 (steady) or Algorithm 3 (unsteady) applied once."""
    It = I.T.tocsr()
    ne, s = mesh_c.ne, ops["s"]
    M2 = (It @ ops["M"] @ I).tocsr()
    M2inv = blockdiag_inverse(M2, ne, s)
    out = dict(mesh=mesh_c, s=s, M=M2)
    out["Mmu"] = (It @ ops["Mmu"] @ I).tocsr()
    out["G"] = [(M2inv @ It @ ops["M"] @ Gk @ I).tocsr() for Gk in ops["G"]]
    out["Et"] = (0.5 * (It @ ops["Et"] @ I)).tocsr()
    if unsteady:
        out["Mrho"] = (It @ ops["Mrho"] @ I).tocsr()
        out["Emu"] = (2.0 * (It @ ops["Emu"] @ I)).tocsr()
        out["Erho"] = (0.5 * (It @ ops["Erho"] @ I)).tocsr()
        out["E"] = combine_pressure_penalty(out["Emu"], out["Erho"], ne, s)
    else:
        out["E"] = (2.0 * (It @ ops["E"] @ I)).tocsr()
    return out


def field_to_element_perm(ne, s, nvar):
    """Permutation matrix P with (P x_field)[e*nvar*s + v*s + a] = x_field[v*ne*s + e*s + a]."""
    e, v, a = np.meshgrid(np.arange(ne), np.arange(nvar), np.arange(s), indexing="ij")
    new = (e * nvar * s + v * s + a).ravel()
    old = (v * ne * s + e * s + a).ravel()
    n = ne * s * nvar
    return sp.csr_matrix((np.ones(n), (new, old)), shape=(n, n))


def stokes_operator(ops, gamma, delta=None):
    """The symmetric saddle-point operator of eq. (blockform) / (timedep2),
    field-major [u_1 .. u_d, p]."""
    G = ops["G"]
    d = len(G)
    M, Mmu = ops["M"], ops["Mmu"]
    ne, s = ops["mesh"].ne, ops["s"]
    Minv = blockdiag_inverse(M, ne, s)
    lap = sum(Gk.T @ Mmu @ Gk for Gk in G) + ops["Et"]
    if delta is not None:
        lap = lap + (1.0 / delta) * ops["Mrho"]
    Gcal = [-(Minv @ Gi.T @ M) for Gi in G]
    blocks = [[None] * (d + 1) for _ in range(d + 1)]
    for i in range(d):
        for j in range(d):
            Aij = gamma * (G[j].T @ Mmu @ G[i])
            if i == j:
                Aij = Aij + lap
            blocks[i][j] = Aij
        blocks[i][d] = M @ Gcal[i]
        blocks[d][i] = Gcal[i].T @ M
    blocks[d][d] = -ops["E"]
    return sp.bmat(blocks, format="csr")


def sqrt_mu_scaling(ops, d):
    """Section 5.6 diagonal scaling: per element mu_E^{-1/2} on the velocity
    unknowns and mu_E^{1/2} on the pressure unknowns, with mu_E the element
    mean of mu (M_mu(E)[0,0] / M(E)[0,0], mode 0 being the constant).  Returned
    as the element-major diagonal."""
    ne, s = ops["mesh"].ne, ops["s"]
    Mmu = diag_blocks(ops["Mmu"], ne, s)[:, 0, 0]
    M = diag_blocks(ops["M"], ne, s)[:, 0, 0]
    mu_e = Mmu / M
    dv = np.repeat(mu_e ** -0.5, d * s).reshape(ne, d * s)
    dp = np.repeat(mu_e ** 0.5, s).reshape(ne, s)
    return np.concatenate([dv, dp], axis=1).ravel()


class Level:
    """One level of the hierarchy: the element-major Stokes operator (scaled
    by D A D when the sqrt(mu) scaling is on, every level with its own mu_E)
    and the data the smoother and transfers need."""

    def __init__(self, ops, gamma, delta, d, scale=False):
        self.ops = ops
        self.mesh = ops["mesh"]
        self.s = ops["s"]
        self.nvar = d + 1
        self.nb = self.nvar * self.s
        self.ne = self.mesh.ne
        Afield = stokes_operator(ops, gamma, delta)
        self.P = field_to_element_perm(self.ne, self.s, self.nvar)
        self.A = (self.P @ Afield @ self.P.T).tocsr()
        self.D = None
        if scale:
            self.D = sqrt_mu_scaling(ops, d)
            Dm = sp.diags(self.D)
            self.A = (Dm @ self.A @ Dm).tocsr()
        self.A.sum_duplicates()
        self.A.sort_indices()


def build_hierarchy(prob, max_levels=None):
    """Fine operators (Appendix A), then recursive coarsening (Appendix B)."""
    unsteady = prob.delta is not None
    scale = bool(prob.scale_mu)
    ops = fine_operators(prob)
    levels = [Level(ops, prob.gamma, prob.delta, prob.d, scale)]
    injections = []
    while True:
        mesh = ops["mesh"]
        if any(n % 2 == 1 or n <= 2 for n in mesh.n):
            break
        if max_levels is not None and len(levels) >= max_levels:
            break
        nc = [n // 2 for n in mesh.n]
        chi_c = None
        if mesh.chi is not None:
            # Same-phase agglomeration (Section 3): a coarse cell exists only if
            # all of its children belong to one phase; otherwise stop here.
            parent = ((mesh.idx // 2) * np.asarray([int(np.prod(nc[:k])) for k in range(mesh.d)])).sum(axis=1)
            nec = int(np.prod(nc))
            lo_ph = np.full(nec, 10 ** 9)
            hi_ph = np.full(nec, -1)
            np.minimum.at(lo_ph, parent, mesh.chi)
            np.maximum.at(hi_ph, parent, mesh.chi)
            if np.any(lo_ph != hi_ph):
                break
            chi_c = lo_ph
        mesh_c = Mesh(mesh.d, nc, mesh.lo, mesh.hi, mesh.bc, chi=chi_c)
        I = injection(mesh, mesh_c, prob.p)
        ops = coarsen(ops, I, mesh_c, unsteady)
        lev = Level(ops, prob.gamma, prob.delta, prob.d, scale)
        # Full (all variables) injection in element-major order.
        Ifull_field = sp.block_diag([I] * (prob.d + 1), format="csr")
        injections.append((levels[-1].P @ Ifull_field @ lev.P.T).tocsr())
        levels.append(lev)
    return levels, injections
