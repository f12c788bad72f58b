"""Tensor-product Legendre basis and Gauss quadrature (oracle).

Section 2 and Appendix A fix the space Q_p(E) of tensor-product polynomials of
one-dimensional degree p on each element, but not the basis.  Reading: on the
reference interval [-1, 1] the 1-D basis is psi_l = sqrt(2l+1) P_l (Legendre),
so that int_{-1}^{1} psi_m psi_l = 2 delta_ml and the element mass matrix is
|E| times the identity.  Modes are ordered lexicographically with the x index
fastest: a = a_0 + (p+1) a_1 + (p+1)^2 a_2.

Quadrature: Gauss-Legendre (numpy.polynomial.legendre.leggauss).
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gauss(q):
    """q-point Gauss-Legendre rule on [-1, 1]."""
    return npleg.leggauss(q)


def psi(p, xi):
    """Table [len(xi), p+1] of psi_l(xi) = sqrt(2l+1) P_l(xi)."""
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    out = np.empty((xi.size, p + 1))
    for l in range(p + 1):
        c = np.zeros(l + 1)
        c[l] = 1.0
        out[:, l] = np.sqrt(2 * l + 1) * npleg.legval(xi, c)
    return out


def dpsi(p, xi):
    """Table [len(xi), p+1] of d psi_l / d xi."""
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    out = np.empty((xi.size, p + 1))
    for l in range(p + 1):
        c = np.zeros(l + 1)
        c[l] = 1.0
        out[:, l] = np.sqrt(2 * l + 1) * npleg.legval(xi, npleg.legder(c))
    return out


def mass_1d(p):
    """int psi_m psi_l over [-1, 1]; equals 2 I (used as a check)."""
    x, w = gauss(p + 1)
    P = psi(p, x)
    return P.T @ (w[:, None] * P)


def deriv_1d(p):
    """K[m, l] = int_{-1}^{1} psi_m psi_l' dxi (exact with p+1 points)."""
    x, w = gauss(p + 1)
    return psi(p, x).T @ (w[:, None] * dpsi(p, x))


def trace_1d(p, side):
    """Row vector psi_l(side) for side = -1 or +1."""
    return psi(p, np.array([float(side)]))[0]


def child_1d(p, c):
    """1-D injection matrix of child c (0 = lower half, 1 = upper half):
    fine coefficient m of the coarse mode l restricted to the child,
    P[m, l] = 1/2 int_{-1}^{1} psi_m(xi) psi_l((xi + 2c - 1)/2) dxi."""
    x, w = gauss(p + 1)
    return 0.5 * psi(p, x).T @ (w[:, None] * psi(p, (x + 2 * c - 1) / 2.0))


def kron_axes(mats):
    """Kronecker product of per-axis matrices mats[0..d-1] with axis 0 the
    fastest index: kron(mats[d-1], ..., mats[0])."""
    out = np.ones((1, 1))
    for m in mats:
        out = np.kron(m, out)
    return out


def axis_op(d, p, k, T):
    """Operator acting with T on axis k and the identity on the other axes."""
    return kron_axes([T if j == k else np.eye(p + 1) for j in range(d)])


def tensor_rule(d, q):
    """Tensor Gauss rule on [-1,1]^d: points [q^d, d] (axis 0 fastest), weights."""
    x, w = gauss(q)
    pts = np.zeros((q ** d, d))
    wts = np.ones(q ** d)
    idx = np.arange(q ** d)
    for k in range(d):
        ik = (idx // q ** k) % q
        pts[:, k] = x[ik]
        wts *= w[ik]
    return pts, wts


def tensor_basis(d, p, q):
    """Phi[qpt, a] of the tensor basis at the tensor Gauss points."""
    x, _ = gauss(q)
    return kron_axes([psi(p, x)] * d)


def face_rule(d, q, k):
    """Rule on the face orthogonal to axis k: points [q^(d-1), d] with the
    axis-k coordinate set to 0 (caller fills it), weights on [-1,1]^(d-1)."""
    if d == 1:
        return np.zeros((1, 1)), np.ones(1)
    sub, w = tensor_rule(d - 1, q)
    pts = np.zeros((sub.shape[0], d))
    others = [j for j in range(d) if j != k]
    for t, j in enumerate(others):
        pts[:, j] = sub[:, t]
    return pts, w


def face_basis(d, p, q, k, side):
    """Phi_F[qpt, a]: tensor basis evaluated on the face xi_k = side at the
    face Gauss points (other axes in increasing order, lower axis fastest)."""
    x, _ = gauss(q)
    mats = []
    for j in range(d):
        mats.append(trace_1d(p, side)[None, :] if j == k else psi(p, x))
    return kron_axes(mats)
