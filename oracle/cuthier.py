"""Multigrid hierarchy on the cut-cell mesh of an embedded circle (oracle).

* Coarse elements by same-phase agglomeration (Section 3): the elements of a
  level are grouped by the parent cell (halved grid) of their anchor cell and
  by phase; each group is one coarse element, anchored at that parent cell.
  The anchor of a fine element is the host cell of its representative piece.
* A coarse element's basis is Q_p on the bounding box of its members' boxes;
  the injection I (Section 3: the coarse function restricted to the fine
  element) maps it onto each member's basis.  A Q_p polynomial on one box is a
  Q_p polynomial on any other, so the restriction is exact and equals the L2
  projection over any region of the member's box; it is taken over the whole
  box, I_f = M_B^{-1} int_B phi_f phi_c^T (B the member's bounding box, a
  tensor Gauss rule with p + 1 points per axis, exact for the degree-2p
  integrand), where the projection over a small cut piece would divide by a
  nearly singular mass matrix.
* Coarse operators by Algorithm 2 (steady) or Algorithm 3 (unsteady;
  hierarchy.coarsen), the Stokes operator of eq. (blockform) / (timedep2) on
  every level; with scale the Section 5.6 scaling D A D on every level, D from
  that level's element mean viscosity.
* The levels halve the grid until it is 2 x 2 cells; the last is the bottom.
* Smoother colouring: deterministic greedy over the structural coupling graph
  (element pairs that some block of the operator joins structurally), elements
  in index order, each the smallest colour unused by an already coloured
  neighbour.  The field operators G_k, E, E~ of a level couple elements one
  face / interface step apart (on a coarse level: groups with members one
  step apart), and the Stokes operator's G^T M G reaches two such steps, so
  the graph is the square of the level's one-step graph.
"""
import types

import numpy as np
import scipy.sparse as sp

from . import basis, cutldg
from .hierarchy import coarsen, field_to_element_perm, sqrt_mu_scaling, stokes_operator


class CutLevel:
    """A level of the cut hierarchy: element boxes and phases, the Stokes
    operator (element-major), and the element colouring."""


def _face_graph(ne, ops):
    intra, bdry, arcs = ops["faces"]
    rows, cols = list(range(ne)), list(range(ne))
    for ea, eb, *_ in intra:
        rows += [ea, eb]
        cols += [eb, ea]
    for em, ep, *_ in arcs:
        rows += [em, ep]
        cols += [ep, em]
    return sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(ne, ne))


def greedy_colours(structure):
    """structure: sparse element x element pattern (nonzero = coupled)."""
    S = structure.tocsr()
    ne = S.shape[0]
    col = np.full(ne, -1, dtype=np.int64)
    for e in range(ne):
        used = {int(col[j]) for j in S.indices[S.indptr[e]:S.indptr[e + 1]] if j != e and col[j] >= 0}
        c = 0
        while c in used:
            c += 1
        col[e] = c
    return col


def build(mesh, p, mu_phase, tau, gamma, nmin=2, rho_phase=None, delta=None, tau0=None, scale=False):
    """Levels [CutLevel] and element-major injections [sparse] of the cut
    hierarchy of the CutMesh `mesh`.  With scale, level l's operator is
    D_l A_l D_l and the transfers stay the plain injection, as on Cartesian
    grids; with one viscosity per phase and same-phase agglomeration a coarse
    element has its members' mu_E, so D_l^{-1} I D_{l+1} = I and the scaled
    and plain transfers agree."""
    unsteady = delta is not None
    ops = cutldg.operators(mesh, p, mu_phase, tau, rho_phase=rho_phase, delta=delta, tau0=tau0)
    els = ops["els"]
    s = ops["s"]
    nvar = 3
    ne = els.ne
    anchor = np.array([mesh.pieces[els.reps[e]]["cell"] for e in range(ne)])
    box_lo, box_hi = els.box_lo.copy(), els.box_hi.copy()
    phase = els.phase.copy()
    G1 = _face_graph(ne, ops)                            # one face / interface step
    structure = ((G1 @ G1) != 0).astype(np.float64)       # blocks of G^T M G reach two steps
    levels, injections = [], []
    n = mesh.n

    def make_level(ops, ne, box_lo, box_hi, phase, structure):
        lev = CutLevel()
        lev.ops, lev.ne, lev.s, lev.nb = ops, ne, s, nvar * s
        lev.box_lo, lev.box_hi, lev.phase = box_lo, box_hi, phase
        Af = stokes_operator(ops, gamma, delta)
        lev.P = field_to_element_perm(ne, s, nvar)
        lev.A = (lev.P @ Af @ lev.P.T).tocsr()
        if scale:
            lev.D = sqrt_mu_scaling(ops, 2)
            Dm = sp.diags(lev.D)
            lev.A = (Dm @ lev.A @ Dm).tocsr()
        else:
            lev.D = None
        lev.A.sum_duplicates()
        lev.structure = structure
        lev.colour = greedy_colours(structure)
        lev.mesh = types.SimpleNamespace(ne=ne, colour=lambda c=lev.colour: c)
        return lev

    levels.append(make_level(ops, ne, box_lo, box_hi, phase, structure))
    fine_phi = lambda e, x: els.phi(e, x)[0]
    while n > nmin:
        n //= 2
        keys = {}
        parent = np.zeros(ne, dtype=np.int64)
        for e in range(ne):
            key = (int(anchor[e][0] // 2), int(anchor[e][1] // 2), int(phase[e]))
            if key not in keys:
                keys[key] = len(keys)
            parent[e] = keys[key]
        order = sorted(keys, key=lambda k: (k[1], k[0], k[2]))     # coarse cells lexicographic, phase
        renum = {keys[k]: i for i, k in enumerate(order)}
        parent = np.array([renum[v] for v in parent])
        nc = len(order)
        c_anchor = np.array([[k[0], k[1]] for k in order])
        c_phase = np.array([k[2] for k in order])
        c_lo = np.full((nc, 2), np.inf)
        c_hi = np.full((nc, 2), -np.inf)
        for e in range(ne):
            c_lo[parent[e]] = np.minimum(c_lo[parent[e]], box_lo[e])
            c_hi[parent[e]] = np.maximum(c_hi[parent[e]], box_hi[e])
        tmp = cutldg.CutElements.__new__(cutldg.CutElements)
        tmp.p = p
        tmp.box_lo, tmp.box_hi = c_lo, c_hi
        coarse_phi = lambda c, x, t=tmp: cutldg.CutElements.phi(t, c, x)[0]
        # scalar injection: fine x coarse, block (f, parent[f]) = M_B^{-1} int_B phi_f phi_c^T
        rows, cols, vals = [], [], []
        for f in range(ne):
            xs, wx = basis.gauss(p + 1)
            gx = 0.5 * (box_lo[f][0] + box_hi[f][0]) + 0.5 * (box_hi[f][0] - box_lo[f][0]) * xs
            gy = 0.5 * (box_lo[f][1] + box_hi[f][1]) + 0.5 * (box_hi[f][1] - box_lo[f][1]) * xs
            X, Y = np.meshgrid(gx, gy, indexing="xy")
            pts = np.stack([X.ravel(), Y.ravel()], axis=1)
            w = np.outer(wx, wx).ravel() * 0.25 * np.prod(box_hi[f] - box_lo[f])
            Pf = fine_phi(f, pts)
            Pc = coarse_phi(parent[f], pts)
            blk = np.linalg.solve(Pf.T @ (w[:, None] * Pf), Pf.T @ (w[:, None] * Pc))
            a = np.arange(s)
            rows.append(np.repeat(f * s + a, s))
            cols.append(np.tile(parent[f] * s + a, s))
            vals.append(blk.ravel())
        I = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(ne * s, nc * s))
        ops = coarsen(ops, I, types.SimpleNamespace(ne=nc), unsteady)
        Pm = sp.csr_matrix((np.ones(ne), (np.arange(ne), parent)), shape=(ne, nc))
        G1 = ((Pm.T @ G1 @ Pm) != 0).astype(np.float64)
        structure = ((G1 @ G1) != 0).astype(np.float64)
        lev = make_level(ops, nc, c_lo, c_hi, c_phase, structure)
        Ifull = sp.block_diag([I] * nvar, format="csr")
        injections.append((levels[-1].P @ Ifull @ lev.P.T).tocsr())
        levels.append(lev)
        # the next coarsening works on this level's elements and boxes
        fine_phi = coarse_phi
        ne, anchor, box_lo, box_hi, phase = nc, c_anchor, c_lo, c_hi, c_phase
    return levels, injections
