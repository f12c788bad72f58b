"""Chebyshev-accelerated block Gauss-Seidel (oracle; test infrastructure only).

The Concluding Remarks name low-degree Chebyshev iterations as a way to
accelerate the Gauss-Seidel smoother, without parameters.  This module states
the published Chebyshev semi-iteration (Golub and Varga; in the form of Saad,
"Iterative Methods for Sparse Linear Systems", the Chebyshev acceleration
algorithm) for the preconditioned operator M^{-1} A, with M the forward
coloured block Gauss-Seidel splitting, so that z = M^{-1} r is one coloured
sweep from a zero guess with right-hand side r:

    r_0 = b - A x_0,  z_0 = M^{-1} r_0,  q_0 = 1 / theta,  d_0 = q_0 z_0
    x_{k+1} = x_k + d_k
    r_{k+1} = b - A x_{k+1},  z_{k+1} = M^{-1} r_{k+1}
    q_{k+1} = 1 / (2 theta - delta^2 q_k)
    d_{k+1} = delta^2 q_{k+1} q_k d_k + 2 q_{k+1} z_{k+1}

for a spectrum of M^{-1} A inside the ellipse with centre theta and foci
theta +- delta.  Saad's recurrence carries rho_k = 1 / (2 sigma - rho_{k-1}),
sigma = theta / delta, and d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1} / delta)
r_{k+1}; with q_k = rho_k / delta every coefficient above is a function of
delta^2, so the iteration stays real for an ellipse symmetric about the real
axis with real foci (delta^2 > 0) or imaginary ones (delta^2 < 0).
`chebyshev_complex` runs Saad's form in complex arithmetic for the pins.

Reading (the paper gives no parameters): on each level the ellipse is fitted
to the eigenvalues mu of M^{-1} A with Re mu >= frac * max Re mu (the part
the smoother must damp; the coarse grid takes the rest, as Chebyshev
smoothers for symmetric problems take [lambda_max / 30, lambda_max]): theta
the midpoint of their real range, semi-axes a = half the real range and
b = their largest |Im mu|, delta^2 = a^2 - b^2.  The eigenvalues are computed
densely, so this reference is for small problems.
"""
import numpy as np

from .multigrid import Multigrid


def chebyshev_iteration(apply_A, apply_Minv, x, b, k, theta, delta2):
    """k steps of the preconditioned Chebyshev iteration from x (in place);
    returns x.  k = 1 with theta = 1 is one preconditioned Richardson step,
    x + M^{-1} (b - A x), i.e. one Gauss-Seidel sweep."""
    if k <= 0:
        return x
    z = apply_Minv(b - apply_A(x))
    q = 1.0 / theta
    d = q * z
    for step in range(k):
        x += d
        if step == k - 1:
            break
        z = apply_Minv(b - apply_A(x))
        qn = 1.0 / (2.0 * theta - delta2 * q)
        d = delta2 * qn * q * d + 2.0 * qn * z
        q = qn
    return x


def chebyshev_complex(apply_A, apply_Minv, x, b, k, theta, delta):
    """Saad's form of the same iteration in complex arithmetic (delta may be
    imaginary); for the pins."""
    x = x.astype(complex)
    r = (b - apply_A(x.real)).astype(complex)
    sigma = theta / delta
    rho = 1.0 / sigma
    d = apply_Minv(r.real).astype(complex) / theta
    for step in range(k):
        x = x + d
        if step == k - 1:
            break
        r = (b - apply_A(x.real)).astype(complex)
        rho_n = 1.0 / (2.0 * sigma - rho)
        d = rho_n * rho * d + (2.0 * rho_n / delta) * apply_Minv(r.real)
        rho = rho_n
    return x


def ellipse_parameters(mu, frac=1.0 / 30.0):
    """(theta, delta^2) of the ellipse around the eigenvalues mu with
    Re mu >= frac * max Re mu (module reading)."""
    mu = np.asarray(mu)
    top = mu.real.max()
    sel = mu[mu.real >= frac * top]
    lo, hi = sel.real.min(), sel.real.max()
    theta = 0.5 * (lo + hi)
    a = 0.5 * (hi - lo)
    b = np.abs(sel.imag).max()
    return float(theta), float(a * a - b * b)


def gs_operator(sm):
    """Dense M^{-1} A of one level's coloured forward Gauss-Seidel splitting
    (column by column: M^{-1} A e_j is one sweep from zero with rhs A e_j)."""
    A = sm.lev.A
    n = A.shape[0]
    out = np.zeros((n, n))
    for j in range(n):
        z = np.zeros(n)
        sm.sweep(z, A[:, j].toarray().ravel())
        out[:, j] = z
    return out


class ChebyshevMultigrid(Multigrid):
    """Algorithm 1 with every smoothing phase of nu Gauss-Seidel sweeps
    replaced by nu steps of the Chebyshev iteration above (nu applications of
    M^{-1}, i.e. nu sweeps, and nu - 1 extra residuals per phase).  params:
    per smoothing level (theta, delta^2); None fits them by ellipse_parameters
    to the dense spectrum of each level's M^{-1} A."""

    def __init__(self, prob, params=None, frac=1.0 / 30.0, **kw):
        super().__init__(prob, **kw)
        if params is None:
            params = [ellipse_parameters(np.linalg.eigvals(gs_operator(sm)), frac) for sm in self.sm]
        self.params = list(params)

    def _smooth(self, l, x, b, nu):
        sm = self.sm[l]
        A = self.levels[l].A
        theta, delta2 = self.params[l]

        def minv(r):
            z = np.zeros_like(r)
            sm.sweep(z, r)
            return z
        return chebyshev_iteration(lambda v: A @ v, minv, x, b, nu, theta, delta2)

    def vcycle(self, x, b, l=0, nu1=None, nu2=None, lexicographic=False):
        nu1 = self.nu1 if nu1 is None else nu1
        nu2 = self.nu2 if nu2 is None else nu2
        if l == len(self.levels) - 1:
            x[:] = self.bottom_solve(b)
            return x
        self._smooth(l, x, b, self.sweeps(nu1, l))
        r2 = self.restrict(l, self.residual(l, x, b))
        x2 = np.zeros_like(r2)
        self.vcycle(x2, r2, l + 1, nu1, nu2)
        x += self.prolong(l, x2)
        self._smooth(l, x, b, self.sweeps(nu2, l))
        return x
