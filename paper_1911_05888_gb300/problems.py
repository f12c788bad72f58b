"""Seeded synthetic problem definitions shared by the tests, the benchmark and the oracle.

This module holds problem *data* only: the mesh box, the polynomial degree, the
boundary types, coefficient fields (viscosity mu, density rho), manufactured
exact solutions and the forcing derived from them, and seeded random vectors.
It contains none of the method's arithmetic (no basis, quadrature, LDG operator,
coarsening or multigrid code), so the CUDA path and the oracle can both draw
their inputs from it without sharing any of the method.

Manufactured solutions follow Appendix C (grid convergence analyses): each
velocity component is a product of shifted sines, and the pressure is a
product of sines scaled by the phase viscosity.  The forcing of the governing
equations, eq. (govern1) / (timedep1), is derived symbolically with sympy:

    rho/delta u - div(mu (grad u + gamma grad u^T)) + grad p = f,   -div u = fdiv.
"""
from __future__ import annotations

import dataclasses
import functools
import math
from typing import Callable, Optional, Sequence

import numpy as np

PERIODIC, DIRICHLET, STRESS = 0, 1, 2
BC_NAMES = {PERIODIC: "periodic", DIRICHLET: "dirichlet", STRESS: "stress"}

# Table 1 of the paper (optimal pressure-penalty prefactor tau), indexed by
# (gamma, d, p).  Stored here as problem data so that callers can pick a tau;
# both implementations receive tau as an explicit input.
TABLE1_TAU = {
    (0, 2, 1): 0.19, (0, 2, 2): 0.10, (0, 2, 3): 0.086, (0, 2, 4): 0.019, (0, 2, 5): 0.031,
    (0, 3, 1): 0.12, (0, 3, 2): 0.088, (0, 3, 3): 0.084,
    (1, 2, 1): 0.14, (1, 2, 2): 0.046, (1, 2, 3): 0.034, (1, 2, 4): 0.0095, (1, 2, 5): 0.011,
    (1, 3, 1): 0.12, (1, 3, 2): 0.039, (1, 3, 3): 0.040,
}
# Table 2: window of tau giving at most 12.5% more iterations than optimal.
TABLE2_WINDOW = {
    (0, 2, 1): (0.15, 0.28), (0, 2, 2): (0.082, 0.12), (0, 2, 3): (0.067, 0.11),
    (0, 2, 4): (0.013, 0.029), (0, 2, 5): (0.021, 0.041),
    (0, 3, 1): (0.061, 0.30), (0, 3, 2): (0.070, 0.11), (0, 3, 3): (0.064, 0.12),
    (1, 2, 1): (0.091, 0.18), (1, 2, 2): (0.040, 0.056), (1, 2, 3): (0.027, 0.043),
    (1, 2, 4): (0.0058, 0.021), (1, 2, 5): (0.0072, 0.020),
    (1, 3, 1): (0.025, 0.19), (1, 3, 2): (0.031, 0.066), (1, 3, 3): (0.021, 0.059),
}


@dataclasses.dataclass
class Problem:
    """A single-phase Cartesian Stokes problem on the box [lo, hi]^d.

    bc[2k] is the boundary type of the low side of axis k, bc[2k+1] of the
    high side (PERIODIC must be set on both sides of an axis).  mu and rho are
    callables of points x[..., d].  delta is None for the steady problem,
    otherwise the time-step-like parameter of eq. (timedep1).
    """
    d: int
    n: tuple
    p: int
    gamma: int
    bc: tuple
    lo: tuple = None
    hi: tuple = None
    mu: Callable = None
    rho: Optional[Callable] = None
    delta: Optional[float] = None
    tau: float = None
    tau0: float = None
    nu1: int = 1
    nu2: int = 1
    exact: "Manufactured" = None
    name: str = ""
    # Multi-phase (grid-aligned phases): phase(x) -> phase index 1..P of the
    # points x[..., d] (elements never straddle an interface); mu_phase[c-1]
    # is the viscosity of phase c; scale_mu applies the sqrt(mu) diagonal
    # scaling of the Stokes operator.
    phase: Optional[Callable] = None
    mu_phase: Optional[Sequence[float]] = None
    scale_mu: bool = False

    def __post_init__(self):
        if self.lo is None:
            self.lo = (0.0,) * self.d
        if self.hi is None:
            self.hi = (1.0,) * self.d
        if self.mu is None:
            self.mu = lambda x: np.ones(x.shape[:-1])
        if self.tau is None:
            self.tau = TABLE1_TAU[(self.gamma, self.d, self.p)]
        if self.tau0 is None:
            self.tau0 = 0.5 * self.p
        self.n = tuple(int(v) for v in self.n)
        for k in range(self.d):
            a, b = self.bc[2 * k], self.bc[2 * k + 1]
            if (a == PERIODIC) != (b == PERIODIC):
                raise ValueError("periodic must be set on both sides of an axis")

    @property
    def nb(self):
        return (self.d + 1) * (self.p + 1) ** self.d

    @property
    def n_elements(self):
        return int(np.prod(self.n))

    @property
    def n_dofs(self):
        return self.n_elements * self.nb

    def with_(self, **kw):
        return dataclasses.replace(self, **kw)


# ---------------------------------------------------------------------------
# Manufactured solutions (Appendix C and the workload shapes)
# ---------------------------------------------------------------------------

class Manufactured:
    """Exact (u, p) with the forcing (f, fdiv), Dirichlet data g = u and stress
    data h = mu (grad u + gamma grad u^T) n - p n, evaluated numerically from a
    sympy expression tree."""

    def __init__(self, d, u_exprs, p_expr, mu_expr, gamma, rho_expr=None, delta=None):
        import sympy as sp
        xs = sp.symbols("x0:%d" % d)
        self.d = d
        self.gamma = gamma
        u = [e(xs) for e in u_exprs]
        pe = p_expr(xs)
        mu = mu_expr(xs)
        grad = [[sp.diff(u[i], xs[j]) for j in range(d)] for i in range(d)]
        tau = [[grad[i][j] + gamma * grad[j][i] for j in range(d)] for i in range(d)]
        sig = [[mu * tau[i][j] - (pe if i == j else 0) for j in range(d)] for i in range(d)]
        f = []
        for i in range(d):
            fi = -sum(sp.diff(mu * tau[i][j], xs[j]) for j in range(d)) + sp.diff(pe, xs[i])
            if delta is not None:
                fi = fi + rho_expr(xs) / delta * u[i]
            f.append(fi)
        fdiv = -sum(sp.diff(u[i], xs[i]) for i in range(d))
        lam = lambda e: sp.lambdify([xs], e, "numpy")
        self._u = [lam(e) for e in u]
        self._p = lam(pe)
        self._f = [lam(e) for e in f]
        self._fdiv = lam(fdiv)
        self._sig = [[lam(sig[i][j]) for j in range(d)] for i in range(d)]
        self._mu = lam(mu)

    @staticmethod
    def _ev(fn, x):
        x = np.asarray(x, dtype=np.float64)
        cols = [x[..., k] for k in range(x.shape[-1])]
        out = fn(cols)
        return np.broadcast_to(np.asarray(out, dtype=np.float64), x.shape[:-1]).copy()

    def u(self, x):
        return np.stack([self._ev(g, x) for g in self._u], axis=-1)

    def p(self, x):
        return self._ev(self._p, x)

    def f(self, x):
        return np.stack([self._ev(g, x) for g in self._f], axis=-1)

    def fdiv(self, x):
        return self._ev(self._fdiv, x)

    def mu(self, x):
        return self._ev(self._mu, x)

    def stress(self, x, nrm):
        """sigma . n at points x with (constant) unit normal nrm."""
        out = np.zeros(np.asarray(x).shape[:-1] + (self.d,))
        for i in range(self.d):
            for j in range(self.d):
                if nrm[j] != 0.0:
                    out[..., i] += self._ev(self._sig[i][j], x) * nrm[j]
        return out


def _sin(v):
    import sympy as sp
    return sp.sin(2 * sp.pi * v)


def _cos(v):
    import sympy as sp
    return sp.cos(2 * sp.pi * v)


def paper_solution(d, gamma, mu_expr=None, rho_expr=None, delta=None, mu_scale=1.0):
    """Appendix C: u_i = prod_j sin 2pi(x_j - 0.2 i), p = mu_chi prod_j sin 2pi(x_j + 0.2)
    (single phase, chi = 1; components i = 1..d)."""
    import sympy as sp
    if mu_expr is None:
        mu_expr = lambda xs: sp.Integer(1)
    u_exprs = []
    for i in range(1, d + 1):
        u_exprs.append(lambda xs, i=i: sp.Mul(*[_sin(xs[j] - sp.Rational(i, 5)) for j in range(d)]))
    p_expr = lambda xs: mu_scale * sp.Mul(*[_sin(xs[j] + sp.Rational(1, 5)) for j in range(d)])
    return Manufactured(d, u_exprs, p_expr, mu_expr, gamma, rho_expr, delta)


def divfree_solution_2d(gamma=0, mu_expr=None):
    """The divergence-free pair u = (sin2pi x cos2pi y, -cos2pi x sin2pi y),
    p = sin2pi x sin2pi y (periodic 16x16 workload)."""
    import sympy as sp
    if mu_expr is None:
        mu_expr = lambda xs: sp.Integer(1)
    u_exprs = [lambda xs: _sin(xs[0]) * _cos(xs[1]), lambda xs: -_cos(xs[0]) * _sin(xs[1])]
    p_expr = lambda xs: _sin(xs[0]) * _sin(xs[1])
    return Manufactured(2, u_exprs, p_expr, mu_expr, gamma)


def timeperiodic_solution_3d(t, omega, re, rho=1.0, delta=None):
    """3D periodic flow scaled by cos(omega t): u = cos(wt)(sin x cos y cos z,
    -cos x sin y cos z, 0), p = cos(wt) sin x sin y sin z (2 pi periods)."""
    import sympy as sp
    c = math.cos(omega * t)
    u_exprs = [lambda xs: c * _sin(xs[0]) * _cos(xs[1]) * _cos(xs[2]),
               lambda xs: -c * _cos(xs[0]) * _sin(xs[1]) * _cos(xs[2]),
               lambda xs: sp.Integer(0) * xs[0]]
    p_expr = lambda xs: c * _sin(xs[0]) * _sin(xs[1]) * _sin(xs[2])
    mu_expr = lambda xs: sp.Float(1.0 / re)
    rho_expr = lambda xs: sp.Float(rho)
    return Manufactured(3, u_exprs, p_expr, mu_expr, 0, rho_expr, delta)


class MultiPhaseManufactured:
    """Appendix C manufactured solution per phase: u_i = prod_j sin 2pi(x_j -
    0.2 i - 0.25(chi-1)), p = mu_chi prod_j sin 2pi(x_j + 0.2 - 0.25(chi-1)),
    with the phase chi of each point; jump data g_ij = u_i - u_j and
    h_ij = sigma_i n - sigma_j n on an interface with normal n from phase i
    (the lower index) into phase j."""

    def __init__(self, d, gamma, mu_phase, phase):
        import sympy as sp
        self.d, self.gamma, self.phase = d, gamma, phase
        self.sol = []
        for c, muc in enumerate(mu_phase, start=1):
            sh = sp.Rational(1, 4) * (c - 1)
            u_exprs = [lambda xs, i=i, sh=sh: sp.Mul(*[_sin(xs[j] - sp.Rational(i, 5) - sh) for j in range(d)])
                       for i in range(1, d + 1)]
            p_expr = lambda xs, sh=sh, muc=muc: sp.Float(muc) * sp.Mul(*[_sin(xs[j] + sp.Rational(1, 5) - sh)
                                                                         for j in range(d)])
            self.sol.append(Manufactured(d, u_exprs, p_expr, lambda xs, muc=muc: sp.Float(muc), gamma))

    def _per_phase(self, name, x, *args, chi=None):
        x = np.asarray(x, dtype=np.float64)
        chi = self.phase(x) if chi is None else np.broadcast_to(chi, x.shape[:-1])
        out = None
        for c, sol in enumerate(self.sol, start=1):
            m = chi == c
            if not np.any(m):
                continue
            v = getattr(sol, name)(x[m], *args)
            if out is None:
                out = np.zeros(x.shape[:-1] + v.shape[1:])
            out[m] = v
        return out

    def u(self, x, chi=None):
        return self._per_phase("u", x, chi=chi)

    def p(self, x, chi=None):
        return self._per_phase("p", x, chi=chi)

    def f(self, x, chi=None):
        return self._per_phase("f", x, chi=chi)

    def fdiv(self, x, chi=None):
        return self._per_phase("fdiv", x, chi=chi)

    def stress(self, x, nrm, chi=None):
        return self._per_phase("stress", x, nrm, chi=chi)

    def jumps(self, x, nrm, chi_minus, chi_plus):
        """(g, h) on interface points x with normal nrm from chi_minus to chi_plus."""
        g = self.u(x, chi=chi_minus) - self.u(x, chi=chi_plus)
        h = self.stress(x, nrm, chi=chi_minus) - self.stress(x, nrm, chi=chi_plus)
        return g, h


@dataclasses.dataclass
class CutProblem:
    """Two-phase Stokes problem on the unit square cut by an embedded circle
    (Section 5's curved interface; the bubble configurations of Section 6):
    phase 1 inside the circle, phase 2 outside, Dirichlet data on the box,
    velocity and stress jumps on the circle from the per-phase manufactured
    solution of Appendix C (MultiPhaseManufactured).  With rho_phase and delta
    the unsteady problem of eq. (timedep1); its forcing adds rho/delta u.
    With inside_only and one viscosity, the disc alone (Section 5's curved
    domain) with Dirichlet data from the same solution on the circle."""
    n: int = 128
    p: int = 3
    gamma: int = 1
    mu_phase: Sequence[float] = (1e-3, 1.0)
    rho_phase: Optional[Sequence[float]] = None
    delta: Optional[float] = None
    centre: Sequence[float] = (0.5, 0.5)
    radius: float = 0.25
    nu1: int = 3
    nu2: int = 3
    tau: Optional[float] = None
    tau0: Optional[float] = None
    scale_mu: bool = True
    inside_only: bool = False   # the disc alone (one phase, Dirichlet data on the circle)

    def __post_init__(self):
        if self.tau is None:
            self.tau = TABLE1_TAU[(self.gamma, 2, self.p)]
        if self.tau0 is None:
            self.tau0 = 0.5 * self.p
        c, r = np.asarray(self.centre, dtype=np.float64), float(self.radius)
        self.phase = lambda x: np.where(np.sqrt(((np.asarray(x) - c) ** 2).sum(-1)) < r, 1, 2)
        self.exact = MultiPhaseManufactured(2, self.gamma, list(self.mu_phase), self.phase)
        self.d = 2

    @property
    def unsteady(self):
        return self.delta is not None and self.delta > 0

    def forcing(self, x, chi):
        """(f_1, f_2, fdiv) at points x of phase chi, with rho/delta u for the
        unsteady problem."""
        f = self.exact.f(x, chi=chi)
        if self.unsteady:
            rho = np.asarray(self.rho_phase, dtype=np.float64)[np.asarray(chi) - 1]
            f = f + (rho / self.delta)[:, None] * self.exact.u(x, chi=chi)
        return np.concatenate([f, self.exact.fdiv(x, chi=chi)[:, None]], axis=1)


def square_interface(d=2, n=16, p=2, mu_inner=1e-3, mu_outer=1.0, nu=(3, 3), tau=None, scale_mu=True,
                     bc=None):
    """Multi-phase test of Section 5.6: phase 1 = (1/4, 3/4)^d with viscosity
    mu_inner, phase 2 outside with mu_outer, viscous-stress form, periodic."""
    mu_phase = [mu_inner, mu_outer]

    def phase(x):
        x = np.asarray(x, dtype=np.float64)
        inside = np.all((x > 0.25) & (x < 0.75), axis=-1)
        return np.where(inside, 1, 2)

    def mu(x):
        return np.where(phase(x) == 1, mu_inner, mu_outer).astype(np.float64)

    ex = MultiPhaseManufactured(d, 1, mu_phase, phase)
    return Problem(d=d, n=(n,) * d, p=p, gamma=1, bc=tuple(bc or (PERIODIC,) * (2 * d)), mu=mu, tau=tau,
                   nu1=nu[0], nu2=nu[1], exact=ex, phase=phase, mu_phase=mu_phase, scale_mu=scale_mu,
                   name="%dd-square-interface-n%d-p%d-ratio%g" % (d, n, p, mu_inner / mu_outer))


def mu_variable_2d(seed=0, n_extra=0):
    """Viscosity mu = 1 + 0.9 sin2pi x cos2pi y plus optional seeded extra modes
    of amplitude <= 0.05 (kept >= 0.05 overall)."""
    import sympy as sp
    rng = np.random.default_rng(seed)
    extra = [(int(rng.integers(1, 4)), int(rng.integers(1, 4)), float(rng.uniform(-0.05, 0.05)))
             for _ in range(n_extra)]

    def expr(xs):
        e = 1 + sp.Rational(9, 10) * _sin(xs[0]) * _cos(xs[1])
        for kx, ky, a in extra:
            e = e + a * sp.sin(2 * sp.pi * kx * xs[0]) * sp.sin(2 * sp.pi * ky * xs[1])
        return e
    return expr


# ---------------------------------------------------------------------------
# Workload shapes
# ---------------------------------------------------------------------------

def periodic_standard_2d(n=16, p=2, nu=(1, 1), tau=None):
    """Steady standard form, periodic unit square, mu = 1, divergence-free pair."""
    ex = divfree_solution_2d(0)
    return Problem(d=2, n=(n, n), p=p, gamma=0, bc=(PERIODIC,) * 4, tau=tau,
                   nu1=nu[0], nu2=nu[1], exact=ex, name="2d-periodic-standard-n%d-p%d" % (n, p))


def stress_variable_mu_2d(n=256, p=3, nu=(1, 1), tau=None, seed=0):
    """Steady viscous-stress form, Dirichlet on three sides and a stress
    condition on the top side (y = 1), mu = 1 + 0.9 sin2pi x cos2pi y."""
    mu_expr = mu_variable_2d(seed)
    ex = paper_solution(2, 1, mu_expr=mu_expr)
    return Problem(d=2, n=(n, n), p=p, gamma=1, bc=(DIRICHLET, DIRICHLET, DIRICHLET, STRESS),
                   mu=ex.mu, tau=tau, nu1=nu[0], nu2=nu[1], exact=ex,
                   name="2d-stress-varmu-n%d-p%d" % (n, p))


def generic(d, n, p, gamma, bc, mu=None, tau=None, nu=(1, 1), rho=None, delta=None, exact=None):
    return Problem(d=d, n=(n,) * d if np.isscalar(n) else tuple(n), p=p, gamma=gamma, bc=tuple(bc),
                   mu=mu, rho=rho, delta=delta, tau=tau, nu1=nu[0], nu2=nu[1], exact=exact)


def unsteady_periodic_3d(n=48, p=2, re=1.0, t=0.0, nu=(1, 1), tau=None, omega=None):
    """Unsteady standard form on the periodic cube, rho = 1, mu = 1/Re,
    delta = 0.1 h (CFL about 0.1, as in the single-phase unsteady tests)."""
    h = 1.0 / n
    delta = 0.1 * h
    if omega is None:
        omega = 2 * math.pi / (16 * delta)
    ex = timeperiodic_solution_3d(t, omega, re, 1.0, delta)
    return Problem(d=3, n=(n,) * 3, p=p, gamma=0, bc=(PERIODIC,) * 6,
                   mu=lambda x: np.full(x.shape[:-1], 1.0 / re),
                   rho=lambda x: np.ones(x.shape[:-1]), delta=delta, tau=tau,
                   nu1=nu[0], nu2=nu[1], exact=ex, name="3d-unsteady-periodic-n%d-p%d-re%g" % (n, p, re))


def mu_contrast_2d(seed, contrast):
    """Smooth seeded viscosity mu = exp(a s(x, y)) with s a normalised sum of
    three Fourier modes (|s| <= 1) and a = ln(contrast) / 2, so that
    max mu / min mu <= contrast."""
    import sympy as sp
    rng = np.random.default_rng(seed)
    modes = [(int(rng.integers(1, 3)), int(rng.integers(1, 3)), float(rng.uniform(0.2, 1.0)),
              float(rng.uniform(0, 1))) for _ in range(3)]
    total = sum(m[2] for m in modes)
    a = math.log(contrast) / 2

    def expr(xs):
        s = 0
        for kx, ky, amp, ph in modes:
            s = s + amp / total * sp.sin(2 * sp.pi * (kx * xs[0] + ph)) * sp.cos(2 * sp.pi * ky * xs[1])
        return sp.exp(a * s)
    return expr


def unsteady_stress_2d(n=64, p=3, seed=0, contrast=100.0, nu=(3, 3), tau=None):
    """2D unsteady viscous-stress form (eq. timedep1 with gamma = 1): Dirichlet
    on three sides and a stress condition on the top, rho = 1, delta = 0.1 h,
    seeded smooth viscosity with max / min <= contrast (mu_contrast_2d), the
    manufactured solution of Appendix C with its mass term."""
    import sympy as sp
    h = 1.0 / n
    delta = 0.1 * h
    mu_expr = mu_contrast_2d(seed, contrast)
    ex = paper_solution(2, 1, mu_expr=mu_expr, rho_expr=lambda xs: sp.Integer(1), delta=delta)
    return Problem(d=2, n=(n, n), p=p, gamma=1, bc=(DIRICHLET, DIRICHLET, DIRICHLET, STRESS),
                   mu=ex.mu, rho=lambda x: np.ones(x.shape[:-1]), delta=delta, tau=tau,
                   nu1=nu[0], nu2=nu[1], exact=ex, name="2d-unsteady-stress-n%d-p%d-seed%d" % (n, p, seed))


def serving_mix(count=64, seed=0, sizes=(32, 64, 128, 256), degrees=(2, 3), contrast=100.0):
    """The batched serving mix: `count` unsteady viscous-stress problems with
    mesh sizes and degrees drawn uniformly (seeded) and viscosity contrasts
    up to `contrast` (problem i uses viscosity seed 1000 + i)."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(sizes, count)
    ps = rng.choice(degrees, count)
    return [unsteady_stress_2d(n=int(ns[i]), p=int(ps[i]), seed=1000 + i, contrast=contrast) for i in range(count)]


# ---------------------------------------------------------------------------
# Seeded vectors
# ---------------------------------------------------------------------------

def random_vector(n_elements, nb, seed, nrhs=1, dtype=np.float64):
    """Uniform(-1, 1) element-blocked vector [n_elements][nb] (or
    [n_elements][nb][nrhs])."""
    rng = np.random.default_rng(seed)
    shape = (n_elements, nb) if nrhs == 1 else (n_elements, nb, nrhs)
    return rng.uniform(-1.0, 1.0, size=shape).astype(dtype)
