"""LDG operators on the cut-cell mesh of an embedded circle (oracle).

Appendix A on the merged elements of cutcell.CutMesh, the same operators as
ldg.py with every integral taken by the cut-cell quadrature:

  * element basis: the tensor Legendre basis Q_p of basis.py on the element's
    bounding box (the hull of its pieces' bounding boxes, cutcell.piece_box;
    an uncut cell's box is the cell), so that the element mass matrix
    M_E = int_E phi_a phi_b is a dense block, not |E| I;
  * G_k = M^{-1}(B_k + L_k): the broken derivative plus the lift of eq. (gsum)
    -- on an intraphase face (axis-aligned, normal +e_k from the left element
    to the right one) into the right (+) element's rows; on a Dirichlet face
    -int u^- v^- n_k; on the circle (normal out of the circle, from phase 1 =
    the - side into phase 2) split (1 - lambda) into the - element and lambda
    into the + element with the viscosity-upwinded lambda of eq.
    (viscosityupwind);
  * E~ (eq. Epenalty): tau_bdry = 10 p mu / h on Dirichlet faces and
    tau_ij = 3 p min(mu^-, mu^+) / h on the circle; E (eq. eop): tau h / mu on
    intraphase faces; h is the cell width;
  * b = M times the right-hand sides of eqs. (appstokes1)-(appstokes2) with the
    Dirichlet data and the jumps g = u^- - u^+, h = (sigma^- - sigma^+) n on the
    circle, the data terms weighted like the lift.

Faces between two pieces of one merged element are interior to it and carry
no term.  Unknowns are numbered [variable][element][mode] (field-major, as in
ldg.py).
"""
import types

import numpy as np
import scipy.sparse as sp

from . import basis, cutcell
from .hierarchy import blockdiag_inverse
from .ldg import _Acc


class CutElements:
    """The merged elements of a CutMesh: pieces, host cells, bounding box
    (hull of the pieces' boxes), phase, and the basis on the box."""

    def __init__(self, mesh, p):
        self.mesh, self.p, self.d = mesh, p, 2
        self.s = (p + 1) ** 2
        self.reps = sorted(set(mesh.element))
        self.index = {rep: e for e, rep in enumerate(self.reps)}
        self.ne = len(self.reps)
        self.of_piece = np.array([self.index[mesh.element[k]] for k in range(len(mesh.pieces))])
        self.pieces = [[] for _ in range(self.ne)]
        for k in range(len(mesh.pieces)):
            self.pieces[self.of_piece[k]].append(k)
        self.phase = np.array([mesh.pieces[self.reps[e]]["phase"] for e in range(self.ne)])
        self.box_lo = np.zeros((self.ne, 2))
        self.box_hi = np.zeros((self.ne, 2))
        for e in range(self.ne):
            self.box_lo[e] = np.min([mesh.pieces[k]["box"][0] for k in self.pieces[e]], axis=0)
            self.box_hi[e] = np.max([mesh.pieces[k]["box"][1] for k in self.pieces[e]], axis=0)

    def phi(self, e, x):
        """(Phi [m, s], [dPhi/dx, dPhi/dy]) of element e at points x [m, 2]."""
        x = np.atleast_2d(x)
        a, b = self.box_lo[e], self.box_hi[e]
        xi = (2 * x - (a + b)) / (b - a)
        P = [basis.psi(self.p, xi[:, k]) for k in range(2)]
        D = [basis.dpsi(self.p, xi[:, k]) * (2.0 / (b[k] - a[k])) for k in range(2)]
        # mode a = a0 + (p+1) a1 (axis 0 fastest)
        Phi = np.einsum("mi,mj->mji", P[0], P[1]).reshape(len(x), -1)
        dx = np.einsum("mi,mj->mji", D[0], P[1]).reshape(len(x), -1)
        dy = np.einsum("mi,mj->mji", P[0], D[1]).reshape(len(x), -1)
        return Phi, [dx, dy]


def faces(mesh, els, q):
    """Intraphase faces (left element, right element, axis, points, weights),
    Dirichlet boundary faces (element, axis, side, points, weights, outward
    normals; axis -1 and side 0 for the circle when it bounds the domain, the
    inside_only mesh) and interface arcs (inside element, outside element,
    points, weights, normals), each from the cut-cell rules."""
    intra, bdry, arcs = [], [], []
    n = mesh.n
    for j in range(n):
        for i in range(n):
            clo = mesh.lo + mesh.h * np.array([i, j])
            for axis in (0, 1):
                o = 1 - axis
                ii, jj = (i + 1, j) if axis == 0 else (i, j + 1)
                fixed = clo[axis] + mesh.h[axis]
                parts = cutcell.face_parts(mesh.circle, clo[o], clo[o] + mesh.h[o], axis, fixed, q)
                for ph, (pts, w) in parts.items():
                    if not len(w):
                        continue
                    if ii < n and jj < n:
                        a = mesh.piece_of.get((i, j, ph))
                        b = mesh.piece_of.get((ii, jj, ph))
                        if a is None or b is None:
                            continue
                        ea, eb = els.of_piece[a], els.of_piece[b]
                        if ea != eb:
                            intra.append((ea, eb, axis, pts, w))
                    else:
                        a = mesh.piece_of.get((i, j, ph))
                        if a is not None:
                            bdry.append((els.of_piece[a], axis, 1, pts, w, _side_normals(axis, 1, len(w))))
                # low boundary sides of the box
                if (axis == 0 and i == 0) or (axis == 1 and j == 0):
                    parts = cutcell.face_parts(mesh.circle, clo[o], clo[o] + mesh.h[o], axis, clo[axis], q)
                    for ph, (pts, w) in parts.items():
                        a = mesh.piece_of.get((i, j, ph))
                        if len(w) and a is not None:
                            bdry.append((els.of_piece[a], axis, -1, pts, w, _side_normals(axis, -1, len(w))))
            if (i, j) in mesh.interface:
                xif, wif, nif = mesh.interface[(i, j)]
                if len(wif):
                    ein = els.of_piece[mesh.piece_of[(i, j, 1)]]
                    out = mesh.piece_of.get((i, j, 2))
                    if out is None:
                        # the circle bounds the domain: a Dirichlet face of the inside element
                        bdry.append((ein, -1, 0, xif, wif, nif))
                    else:
                        arcs.append((ein, els.of_piece[out], xif, wif, nif))
    return intra, bdry, arcs


def _side_normals(axis, side, m):
    nrm = np.zeros((m, 2))
    nrm[:, axis] = side
    return nrm


def operators(mesh, p, mu_phase, tau, q=None, rho_phase=None, delta=None, tau0=None):
    """The Appendix A operators on the cut-cell mesh (Dirichlet on the box, and
    on the circle when the mesh keeps the inside only),
    as a dict like ldg.fine_operators (M, Mmu, G, Et, E, s, mesh with ne).
    With rho_phase and delta the unsteady problem (eq. timedep2): Mrho = rho M
    per element, and on intraphase faces the pressure penalty of eq.
    (taupgeneral), 1 / (h rho / (tau0 delta) + mu / (tau h)), with its two
    limits tau h / mu (Emu) and tau0 delta / (h rho) (Erho) kept for
    Algorithm 3."""
    q = 2 * p + 2 if q is None else q
    unsteady = delta is not None
    if unsteady:
        tau0 = 0.5 * p if tau0 is None else tau0
    els = CutElements(mesh, p)
    s, ne = els.s, els.ne
    hk = mesh.h[0]
    mu = lambda e: mu_phase[els.phase[e] - 1]
    rho = lambda e: rho_phase[els.phase[e] - 1]
    Macc, Mmu_acc, Mrho_acc = _Acc(), _Acc(), _Acc()
    gacc = [_Acc(), _Acc()]
    Et, E, Emu, Erho = _Acc(), _Acc(), _Acc(), _Acc()
    for e in range(ne):
        M = np.zeros((s, s))
        B = [np.zeros((s, s)), np.zeros((s, s))]
        for k in els.pieces[e]:
            pc = mesh.pieces[k]
            Phi, D = els.phi(e, pc["points"])
            w = pc["weights"]
            M += Phi.T @ (w[:, None] * Phi)
            for a in range(2):
                B[a] += Phi.T @ (w[:, None] * D[a])     # rows: test, cols: trial derivative
        Macc.add([e], [e], M[None])
        Mmu_acc.add([e], [e], (mu(e) * M)[None])
        if unsteady:
            Mrho_acc.add([e], [e], (rho(e) * M)[None])
        for a in range(2):
            gacc[a].add([e], [e], B[a][None])
    intra, bdry, arcs = faces(mesh, els, q)
    for ea, eb, axis, pts, w in intra:
        Pa, _ = els.phi(ea, pts)
        Pb, _ = els.phi(eb, pts)
        FF = lambda X, Y: X.T @ (w[:, None] * Y)
        # lift into the + (right) element: int (u^+ - u^-) v^+
        gacc[axis].add([eb], [eb], FF(Pb, Pb)[None])
        gacc[axis].add([eb], [ea], -FF(Pb, Pa)[None])
        if unsteady:
            tmu = tau * hk / mu(ea)
            trho = tau0 * delta / (hk * rho(ea))
            tgen = 1.0 / (hk * rho(ea) / (tau0 * delta) + mu(ea) / (tau * hk))
            coefs = [(E, tgen), (Emu, tmu), (Erho, trho)]
        else:
            coefs = [(E, tau * hk / mu(ea))]
        for acc, tp in coefs:
            for r_, c_, sgn in ((ea, ea, 1), (eb, eb, 1), (ea, eb, -1), (eb, ea, -1)):
                Pr = Pa if r_ == ea else Pb
                Pc = Pa if c_ == ea else Pb
                acc.add([r_], [c_], (sgn * tp * FF(Pr, Pc))[None])
    for e, axis, side, pts, w, nrm in bdry:
        P_, _ = els.phi(e, pts)
        FF = P_.T @ (w[:, None] * P_)
        if axis >= 0:
            gacc[axis].add([e], [e], (-side * FF)[None])
        else:
            # curved Dirichlet boundary: -int u v n_k with the outward normal
            for k in range(2):
                gacc[k].add([e], [e], (-(P_.T @ ((w * nrm[:, k])[:, None] * P_)))[None])
        Et.add([e], [e], (10.0 * p * mu(e) / hk * FF)[None])
    for em, ep, pts, w, nrm in arcs:
        Pm, _ = els.phi(em, pts)
        Pp, _ = els.phi(ep, pts)
        mum, mup = mu(em), mu(ep)
        lam = 0.0 if mum < mup else (1.0 if mum > mup else 0.5)
        for axis in range(2):
            wn = w * nrm[:, axis]
            FF = lambda X, Y: X.T @ (wn[:, None] * Y)
            gacc[axis].add([em], [ep], ((1 - lam) * FF(Pm, Pp))[None])
            gacc[axis].add([em], [em], (-(1 - lam) * FF(Pm, Pm))[None])
            gacc[axis].add([ep], [ep], (lam * FF(Pp, Pp))[None])
            gacc[axis].add([ep], [em], (-lam * FF(Pp, Pm))[None])
        tij = 3.0 * p * min(mum, mup) / hk
        GG = lambda X, Y: X.T @ (w[:, None] * Y)
        Et.add([em], [em], (tij * GG(Pm, Pm))[None])
        Et.add([em], [ep], (-tij * GG(Pm, Pp))[None])
        Et.add([ep], [em], (-tij * GG(Pp, Pm))[None])
        Et.add([ep], [ep], (tij * GG(Pp, Pp))[None])
    M = Macc.csr(ne, s)
    Minv = blockdiag_inverse(M, ne, s)
    G = [(Minv @ g.csr(ne, s)).tocsr() for g in gacc]
    ops = dict(mesh=types.SimpleNamespace(ne=ne), M=M, Mmu=Mmu_acc.csr(ne, s), G=G, Et=Et.csr(ne, s),
               E=E.csr(ne, s), s=s, els=els, faces=(intra, bdry, arcs), Minv=Minv, mu_phase=mu_phase, p=p, q=q)
    if unsteady:
        ops.update(Mrho=Mrho_acc.csr(ne, s), Emu=Emu.csr(ne, s), Erho=Erho.csr(ne, s), delta=delta)
    return ops


def rhs(ops, exact, gamma):
    """b = (b_u, b_p) of eqs. (appstokes1)-(appstokes2) times M on the cut
    mesh, for a per-phase exact solution (exact.u(x, chi=...), .f, .fdiv,
    .stress(x, n, chi=...)); field-major."""
    els, s, p = ops["els"], ops["s"], ops["p"]
    mesh = els.mesh
    ne, hk = els.ne, mesh.h[0]
    mu = lambda e: ops["mu_phase"][els.phase[e] - 1]
    bu = [np.zeros((ne, s)) for _ in range(2)]
    bp = np.zeros((ne, s))
    jg = [[np.zeros((ne, s)) for _ in range(2)] for _ in range(2)]
    for e in range(ne):
        chi = els.phase[e]
        for k in els.pieces[e]:
            pc = mesh.pieces[k]
            Phi, _ = els.phi(e, pc["points"])
            w = pc["weights"]
            f = exact.f(pc["points"], chi=np.full(len(w), chi))
            fd = exact.fdiv(pc["points"], chi=np.full(len(w), chi))
            for i in range(2):
                bu[i][e] += Phi.T @ (w * f[:, i])
            bp[e] += Phi.T @ (w * fd)
    intra, bdry, arcs = ops["faces"]
    for e, axis, side, pts, w, nrm in bdry:
        P_, _ = els.phi(e, pts)
        g = exact.u(pts, chi=np.full(len(w), els.phase[e]))
        tau_d = 10.0 * p * mu(e) / hk
        for i in range(2):
            integ = P_.T @ (w * g[:, i])
            bu[i][e] += tau_d * integ
            if axis >= 0:
                jg[i][axis][e] += side * integ
            else:
                for k in range(2):
                    jg[i][k][e] += P_.T @ (w * nrm[:, k] * g[:, i])
    for em, ep, pts, w, nrm in arcs:
        Pm, _ = els.phi(em, pts)
        Pp, _ = els.phi(ep, pts)
        mum, mup = mu(em), mu(ep)
        lam = 0.0 if mum < mup else (1.0 if mum > mup else 0.5)
        tij = 3.0 * p * min(mum, mup) / hk
        cm, cp = np.full(len(w), els.phase[em]), np.full(len(w), els.phase[ep])
        g = exact.u(pts, chi=cm) - exact.u(pts, chi=cp)
        h = np.zeros_like(g)
        for t in range(len(w)):
            nv = nrm[t]
            h[t] = exact.stress(pts[t:t + 1], nv, chi=cm[:1])[0] - exact.stress(pts[t:t + 1], nv, chi=cp[:1])[0]
        for i in range(2):
            for k in range(2):
                jg[i][k][em] += (1 - lam) * (Pm.T @ (w * nrm[:, k] * g[:, i]))
                jg[i][k][ep] += lam * (Pp.T @ (w * nrm[:, k] * g[:, i]))
            bu[i][em] += lam * (Pm.T @ (w * h[:, i])) + tij * (Pm.T @ (w * g[:, i]))
            bu[i][ep] += (1 - lam) * (Pp.T @ (w * h[:, i])) - tij * (Pp.T @ (w * g[:, i]))
    Minv, Mmu, G = ops["Minv"], ops["Mmu"], ops["G"]
    bu = [b.ravel() for b in bu]
    for i in range(2):
        for j in range(2):
            t = (jg[i][j] + gamma * jg[j][i]).ravel()
            if np.any(t):
                bu[i] -= G[j].T @ (Mmu @ (Minv @ t))
    bp = bp.ravel() + jg[0][0].ravel() + jg[1][1].ravel()
    return np.concatenate(bu + [bp])
