"""Fine-mesh LDG operators for the single-phase Cartesian Stokes problem (oracle).

Follows Appendix A of the paper (LDG methods for the multi-phase Stokes
equations) on a Cartesian grid with one phase:

  * G_k = M^{-1}(B_k + L_k): broken gradient plus the lifting operator L of
    eq. (gsum).  With the one-sided flux u^ = u^- on intraphase faces
    (eq. ustarflux) the lift of an interior face with normal +e_k lands in the
    rows of the right (+) element: int_F (u^+ - u^-) v^+ n_k.  On a velocity
    Dirichlet face the lift is -int_F u^- v^- n; a stress face adds nothing.
  * M is the mass matrix, M_mu (M_rho) the mu- (rho-) weighted mass matrix of
    eq. (sigmaresult) / (timedep2).
  * E~ is the velocity penalty of eq. (Epenalty): tau_{u,0} on intraphase faces
    (zero on Cartesian meshes by default), tau_{u,bdry} = 10 p mu^-/h on
    Dirichlet faces (Appendix A.1 values).
  * E is the pressure penalty of eq. (eop) over intraphase faces only, with
    tau_p = tau h / mu (eq. taueqn) or, for the unsteady problem,
    eq. (taupgeneral); for Algorithm 3 the two parts E_mu, E_rho are also kept.
  * b is M times the right-hand sides of eq. (appstokes1)-(appstokes2).

Readings where the paper is silent (stated once here):
  * h in the penalties is the element width across the face (h_k for a face
    orthogonal to axis k); on a uniform grid this is "the typical element size".
  * mu^-, mu on a face is the mean of mu over the face Gauss points; tau_p is
    constant on each face.
  * M_mu, M_rho and all data integrals use 2p+2 Gauss points per axis.
  * The data term of eq. (appstokes1) is read as
    -sum_j M^{-1} G_j^T M_mu (J_g,ij + gamma J_g,ji): sigma = M^{-1} M_mu tau
    (eq. sigmaresult) carries the mu weight onto J_g; the printed formula omits
    M_mu.
  * In eq. (appstokes2) the sum is over the velocity component index,
    -sum_i G_i u_i.

Scalar unknowns are numbered e*s + a (element e lexicographic with x fastest,
mode a as in basis.py).
"""
import numpy as np
import scipy.sparse as sp

from . import basis
from paper_1911_05888_gb300.problems import PERIODIC, DIRICHLET, STRESS


class Mesh:
    """Cartesian n_0 x ... x n_{d-1} grid on [lo, hi]; chi (optional) is the
    phase of every element (Appendix A: chi(E))."""

    def __init__(self, d, n, lo, hi, bc, chi=None):
        self.d = d
        self.n = tuple(int(v) for v in n)
        self.lo = np.asarray(lo, dtype=np.float64)
        self.hi = np.asarray(hi, dtype=np.float64)
        self.h = (self.hi - self.lo) / np.asarray(self.n, dtype=np.float64)
        self.bc = tuple(bc)
        self.ne = int(np.prod(self.n))
        self.stride = [int(np.prod(self.n[:k])) for k in range(d)]
        e = np.arange(self.ne)
        self.idx = np.stack([(e // self.stride[k]) % self.n[k] for k in range(d)], axis=1)
        self.centre = self.lo + (self.idx + 0.5) * self.h
        self.vol = float(np.prod(self.h))
        self.chi = None if chi is None else np.asarray(chi, dtype=np.int64)

    def periodic(self, k):
        return self.bc[2 * k] == PERIODIC

    def colour_two(self):
        """Two colours (i_1 + ... + i_d) mod 2, the checkerboard: a valid
        colouring of the block GS of Section 3 when the operator couples face
        neighbours only (standard form, gamma = 0, single phase; every level
        of the hierarchy has even n_k or is the unsmoothed bottom)."""
        return self.idx.sum(axis=1) % 2

    def colour(self):
        """Colour of every element for the multi-coloured GS of Section 3.
        Single phase: the parity colouring sum_k (i_k mod 2) 2^k.  With
        phases the interphase lifts couple elements two apart along an axis,
        so a greedy colouring is used instead: elements in order, each takes
        the smallest colour not taken by an already coloured element at any
        offset of the coupling stencil (+-e_k, +-2e_k, +-e_i +- e_j)."""
        if self.chi is None:
            return (self.idx % 2 * (2 ** np.arange(self.d))).sum(axis=1)
        offs = []
        for k in range(self.d):
            for m in (1, 2):
                for sg in (-1, 1):
                    o = [0] * self.d
                    o[k] = sg * m
                    offs.append(o)
        for i in range(self.d):
            for j in range(i + 1, self.d):
                for si in (-1, 1):
                    for sj in (-1, 1):
                        o = [0] * self.d
                        o[i], o[j] = si, sj
                        offs.append(o)
        col = np.full(self.ne, -1, dtype=np.int64)
        for e in range(self.ne):
            used = set()
            for o in offs:
                idx = self.idx[e] + np.asarray(o)
                ok = True
                for k in range(self.d):
                    if idx[k] < 0 or idx[k] >= self.n[k]:
                        if not self.periodic(k):
                            ok = False
                        idx[k] %= self.n[k]
                if ok:
                    j = int((idx * np.asarray(self.stride)).sum())
                    if col[j] >= 0:
                        used.add(int(col[j]))
            c = 0
            while c in used:
                c += 1
            col[e] = c
        return col

    def interior_faces(self, k):
        """(L, R) element pairs sharing a face orthogonal to axis k, the normal
        pointing from L to R (+e_k); periodic wrap faces have L = last, R = first."""
        R = np.nonzero(self.idx[:, k] > 0)[0]
        L = R - self.stride[k]
        if self.periodic(k) and self.n[k] > 1:
            R0 = np.nonzero(self.idx[:, k] == 0)[0]
            L0 = R0 + (self.n[k] - 1) * self.stride[k]
            L = np.concatenate([L, L0])
            R = np.concatenate([R, R0])
        return L, R

    def boundary_faces(self, k, side):
        """Elements touching the low (side=-1) or high (side=+1) boundary of axis k."""
        if self.periodic(k):
            return np.zeros(0, dtype=np.int64)
        i = 0 if side < 0 else self.n[k] - 1
        return np.nonzero(self.idx[:, k] == i)[0]

    def bc_type(self, k, side):
        return self.bc[2 * k + (0 if side < 0 else 1)]

    def face_points(self, elems, k, side, q):
        """Physical Gauss points [len(elems), q^(d-1), d] on the face of each
        element at xi_k = side, and the reference weights."""
        ref, w = basis.face_rule(self.d, q, k)
        ref = ref.copy()
        ref[:, k] = side
        x = self.centre[elems][:, None, :] + 0.5 * self.h[None, None, :] * ref[None, :, :]
        return x, w

    def volume_points(self, q):
        ref, w = basis.tensor_rule(self.d, q)
        x = self.centre[:, None, :] + 0.5 * self.h[None, None, :] * ref[None, :, :]
        return x, w


def blocks_to_csr(ne, s, rows, cols, blocks):
    """Sum s x s blocks placed at (row element, col element) into a CSR matrix."""
    if len(rows) == 0:
        return sp.csr_matrix((ne * s, ne * s))
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    blocks = np.asarray(blocks)
    a = np.arange(s)
    r = (rows[:, None, None] * s + a[None, :, None]) * np.ones((1, 1, s), dtype=np.int64)
    c = (cols[:, None, None] * s + a[None, None, :]) * np.ones((1, s, 1), dtype=np.int64)
    m = sp.coo_matrix((blocks.ravel(), (r.ravel(), c.ravel())), shape=(ne * s, ne * s))
    return m.tocsr()


class _Acc:
    """Accumulates (row element, col element, block) triplets."""

    def __init__(self):
        self.r, self.c, self.b = [], [], []

    def add(self, rows, cols, blocks):
        rows = np.asarray(rows)
        if rows.size == 0:
            return
        blocks = np.asarray(blocks)
        if blocks.ndim == 2:
            blocks = np.broadcast_to(blocks, (rows.size,) + blocks.shape)
        self.r.append(rows)
        self.c.append(np.asarray(cols))
        self.b.append(blocks)

    def csr(self, ne, s):
        if not self.r:
            return sp.csr_matrix((ne * s, ne * s))
        return blocks_to_csr(ne, s, np.concatenate(self.r), np.concatenate(self.c),
                             np.concatenate(self.b))


def interphase_orientation(prob, mesh, L, R):
    """For interphase faces (L left, R right along the axis): the - element
    (lower phase index), the + element, the normal sign sigma (+1 when the
    normal is +e_k) and the viscosity-upwinded lambda of eq. (viscosityupwind)."""
    lowL = mesh.chi[L] < mesh.chi[R]
    minus = np.where(lowL, L, R)
    plus = np.where(lowL, R, L)
    mu_ph = np.asarray(prob.mu_phase, dtype=np.float64)
    mu_m, mu_p = mu_ph[mesh.chi[minus] - 1], mu_ph[mesh.chi[plus] - 1]
    lam = np.where(mu_m < mu_p, 0.0, np.where(mu_m == mu_p, 0.5, 1.0))
    return lowL, minus, plus, lam, mu_m, mu_p


def interphase_faces(prob, mesh, k, L, R, F, g, Et):
    """Interphase faces orthogonal to axis k (Appendix A, eq. gsum and
    eq. Epenalty): lift (1 - lambda)(u^+ - u^-) v^- n + lambda (u^+ - u^-) v^+ n
    and the velocity penalty tau_ij [u][v] with tau_ij = 3 p min(mu^-, mu^+)/h
    (Cartesian value of Appendix A.1); no pressure penalty."""
    if len(L) == 0:
        return
    hk = mesh.h[k]
    area = mesh.vol / hk
    lowL, minus, plus, lam, mu_m, mu_p = interphase_orientation(prob, mesh, L, R)
    tau_ij = 3.0 * prob.p * np.minimum(mu_m, mu_p) / hk
    for orient in (True, False):
        m = lowL == orient
        if not np.any(m):
            continue
        sig = 1.0 if orient else -1.0          # normal from - into +
        sm, sp_ = (1, -1) if orient else (-1, 1)   # face side of the - and + element
        a_m = ((1.0 - lam[m]) * sig * area)[:, None, None]
        a_p = (lam[m] * sig * area)[:, None, None]
        g.add(minus[m], plus[m], a_m * F(k, sm, sp_))
        g.add(minus[m], minus[m], -a_m * F(k, sm, sm))
        g.add(plus[m], plus[m], a_p * F(k, sp_, sp_))
        g.add(plus[m], minus[m], -a_p * F(k, sp_, sm))
        t = (tau_ij[m] * area)[:, None, None]
        Et.add(minus[m], minus[m], t * F(k, sm, sm))
        Et.add(minus[m], plus[m], -t * F(k, sm, sp_))
        Et.add(plus[m], minus[m], -t * F(k, sp_, sm))
        Et.add(plus[m], plus[m], t * F(k, sp_, sp_))


def element_phases(prob, mesh):
    return None if prob.phase is None else np.asarray(prob.phase(mesh.centre), dtype=np.int64)


def fine_operators(prob, quad=None):
    """Assemble the fine-level operators of Appendix A for Problem prob.

    Returns a dict with scipy.sparse CSR matrices M, Mmu, G (list over axes),
    Et (E~), E, and for unsteady problems Mrho, Emu, Erho; plus the mesh."""
    d, p = prob.d, prob.p
    s = (p + 1) ** d
    mesh = Mesh(d, prob.n, prob.lo, prob.hi, prob.bc)
    mesh.chi = element_phases(prob, mesh)
    ne = mesh.ne
    q = 2 * p + 2 if quad is None else quad
    unsteady = prob.delta is not None

    K = basis.deriv_1d(p)
    tp, tm = basis.trace_1d(p, 1), basis.trace_1d(p, -1)
    tr = {1: tp, -1: tm}

    def F(k, sr, sc):
        # [b, a] = psi_{b_k}(sr) psi_{a_k}(sc) delta_perp
        return basis.axis_op(d, p, k, np.outer(tr[sr], tr[sc]))

    # Mass matrices (block diagonal).
    M = sp.identity(ne * s, format="csr") * mesh.vol
    xv, wv = mesh.volume_points(q)
    Phi = basis.tensor_basis(d, p, q)
    jac = mesh.vol / 2 ** d

    def weighted_mass(fun):
        vals = fun(xv)  # [ne, Q]
        blocks = jac * np.einsum("qa,eq,qb->eab", Phi, vals * wv[None, :], Phi)
        e = np.arange(ne)
        return blocks_to_csr(ne, s, e, e, blocks)

    Mmu = weighted_mass(prob.mu)
    Mrho = weighted_mass(prob.rho) if unsteady else None

    def face_mean(fun, elems, k, side):
        x, w = mesh.face_points(elems, k, side, q)
        return (fun(x) * w[None, :]).sum(axis=1) / w.sum()

    MG = []
    Et = _Acc()
    Eacc, Emu_acc, Erho_acc = _Acc(), _Acc(), _Acc()
    for k in range(d):
        hk = mesh.h[k]
        area = mesh.vol / hk
        g = _Acc()
        e = np.arange(ne)
        g.add(e, e, (mesh.vol / hk) * basis.axis_op(d, p, k, K))
        L, R = mesh.interior_faces(k)
        if mesh.chi is not None:
            same = mesh.chi[L] == mesh.chi[R]
            interphase_faces(prob, mesh, k, L[~same], R[~same], F, g, Et)
            L, R = L[same], R[same]
        # Lift of intraphase faces into the + (right) element rows.
        g.add(R, R, area * F(k, -1, -1))
        g.add(R, L, -area * F(k, -1, 1))
        # Pressure penalty over intraphase faces, eq. (eop).
        if len(R):
            mu_f = face_mean(prob.mu, R, k, -1)
            if unsteady:
                rho_f = face_mean(prob.rho, R, k, -1)
                tmu = prob.tau * hk / mu_f
                trho = prob.tau0 * prob.delta / (hk * rho_f)
                tgen = 1.0 / (hk * rho_f / (prob.tau0 * prob.delta) + mu_f / (prob.tau * hk))
                coefs = [(Eacc, tgen), (Emu_acc, tmu), (Erho_acc, trho)]
            else:
                coefs = [(Eacc, prob.tau * hk / mu_f)]
            for acc, tp_ in coefs:
                c = (tp_ * area)[:, None, None]
                acc.add(L, L, c * F(k, 1, 1))
                acc.add(R, R, c * F(k, -1, -1))
                acc.add(L, R, -c * F(k, 1, -1))
                acc.add(R, L, -c * F(k, -1, 1))
        for side in (-1, 1):
            B = mesh.boundary_faces(k, side)
            if len(B) == 0:
                continue
            if mesh.bc_type(k, side) == DIRICHLET:
                g.add(B, B, -side * area * F(k, side, side))
                mu_f = face_mean(prob.mu, B, k, side)
                tau_d = 10.0 * p * mu_f / hk
                Et.add(B, B, (tau_d * area)[:, None, None] * F(k, side, side))
        MG.append(g.csr(ne, s))

    G = [m / mesh.vol for m in MG]  # M^{-1}(B_k + L_k), M = |E| I
    ops = dict(mesh=mesh, M=M, Mmu=Mmu, G=G, Et=Et.csr(ne, s), E=Eacc.csr(ne, s), s=s)
    if unsteady:
        ops.update(Mrho=Mrho, Emu=Emu_acc.csr(ne, s), Erho=Erho_acc.csr(ne, s))
    return ops


def rhs(prob, ops, quad=None):
    """Right-hand side b = (b_u, b_p): M times the right-hand sides of
    eq. (appstokes1) and eq. (appstokes2), field-major [var][e][a]."""
    d, p = prob.d, prob.p
    mesh = ops["mesh"]
    s = ops["s"]
    ne = mesh.ne
    q = 2 * p + 2 if quad is None else quad
    ex = prob.exact
    xv, wv = mesh.volume_points(q)
    Phi = basis.tensor_basis(d, p, q)
    jac = mesh.vol / 2 ** d
    fv = ex.f(xv)  # [ne, Q, d]
    bu = [jac * np.einsum("eq,qa->ea", fv[..., i] * wv[None, :], Phi).ravel() for i in range(d)]
    bp = jac * np.einsum("eq,qa->ea", ex.fdiv(xv) * wv[None, :], Phi).ravel()

    jg = [[np.zeros(ne * s) for _ in range(d)] for _ in range(d)]
    for k in range(d):
        hk = mesh.h[k]
        area = mesh.vol / hk
        for side in (-1, 1):
            B = mesh.boundary_faces(k, side)
            if len(B) == 0:
                continue
            x, w = mesh.face_points(B, k, side, q)
            PhiF = basis.face_basis(d, p, q, k, side)
            fj = area / 2 ** (d - 1)
            nrm = np.zeros(d)
            nrm[k] = side
            kind = mesh.bc_type(k, side)
            if kind == DIRICHLET:
                gv = ex.u(x)  # [nb, Qf, d]
                mu_f = (prob.mu(x) * w[None, :]).sum(axis=1) / w.sum()
                tau_d = 10.0 * p * mu_f / hk
                for i in range(d):
                    integ = fj * np.einsum("fq,qa->fa", gv[..., i] * w[None, :], PhiF)
                    # + int tau_d g_i v  (the -E_{u,g}(0) term)
                    np.add.at(bu[i].reshape(ne, s), B, tau_d[:, None] * integ)
                    # J_g,ik: int g_i n_k v
                    np.add.at(jg[i][k].reshape(ne, s), B, side * integ)
            elif kind == STRESS:
                hv = ex.stress(x, nrm)
                for i in range(d):
                    integ = fj * np.einsum("fq,qa->fa", hv[..., i] * w[None, :], PhiF)
                    np.add.at(bu[i].reshape(ne, s), B, integ)
    if mesh.chi is not None:
        for k in range(d):
            L, R = mesh.interior_faces(k)
            diff = mesh.chi[L] != mesh.chi[R]
            L, R = L[diff], R[diff]
            if len(L) == 0:
                continue
            hk = mesh.h[k]
            area = mesh.vol / hk
            fj = area / 2 ** (d - 1)
            lowL, minus, plus, lam, mu_m, mu_p = interphase_orientation(prob, mesh, L, R)
            tau_ij = 3.0 * p * np.minimum(mu_m, mu_p) / hk
            for orient in (True, False):
                m = lowL == orient
                if not np.any(m):
                    continue
                sig = 1.0 if orient else -1.0
                sm, sp_ = (1, -1) if orient else (-1, 1)
                x, w = mesh.face_points(minus[m], k, sm, q)
                nvec = np.zeros(d)
                nvec[k] = sig
                shp = x.shape[:-1]
                gj, hj = ex.jumps(x.reshape(-1, d), nvec,
                                  np.repeat(mesh.chi[minus[m]], shp[1]), np.repeat(mesh.chi[plus[m]], shp[1]))
                gj, hj = gj.reshape(shp + (d,)), hj.reshape(shp + (d,))
                Pm, Pp = basis.face_basis(d, p, q, k, sm), basis.face_basis(d, p, q, k, sp_)
                lm, lp, tij = (1.0 - lam[m])[:, None], lam[m][:, None], tau_ij[m][:, None]
                for i in range(d):
                    gm = fj * np.einsum("fq,qa->fa", gj[..., i] * w[None, :], Pm)
                    gp = fj * np.einsum("fq,qa->fa", gj[..., i] * w[None, :], Pp)
                    hm = fj * np.einsum("fq,qa->fa", hj[..., i] * w[None, :], Pm)
                    hp = fj * np.einsum("fq,qa->fa", hj[..., i] * w[None, :], Pp)
                    # J_g,ik (eq. gsum), J_h (eq. wworkings) and -E_{u,g}(0) (eq. Epenalty)
                    np.add.at(jg[i][k].reshape(ne, s), minus[m], lm * sig * gm)
                    np.add.at(jg[i][k].reshape(ne, s), plus[m], lp * sig * gp)
                    np.add.at(bu[i].reshape(ne, s), minus[m], lp * hm + tij * gm)
                    np.add.at(bu[i].reshape(ne, s), plus[m], lm * hp - tij * gp)
                    # J_{g.n} (eq. ewv) = sum_i J_g,ii enters b_p below.
    Minv = 1.0 / mesh.vol
    for i in range(d):
        for j in range(d):
            t = jg[i][j] + prob.gamma * jg[j][i]
            if np.any(t):
                bu[i] -= ops["G"][j].T @ (ops["Mmu"] @ (Minv * t))
    for i in range(d):
        bp += jg[i][i]
    return np.concatenate(bu + [bp])
