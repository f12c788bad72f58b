"""Problem-level wrapper over the C ABI: sample the coefficients and data of a
``problems.Problem`` at the library's own quadrature points and drive setup,
right-hand-side assembly, V-cycles and solves.  All arithmetic of the method
runs inside libstokes_mg.so; this module only moves arrays across the ABI."""
import numpy as np

from . import native
from .problems import PERIODIC, DIRICHLET, STRESS


class StokesMG:
    def __init__(self, prob, precision=native.FP64, device=0, nu=None, setup=True, shape=None,
                 colouring=native.COLOURS_AUTO, clusters=False, bottom_max=0):
        self.prob = prob
        self.ctx = native.Context(device)
        d = prob.d
        self.ctx.set_mesh(d, prob.n, prob.lo, prob.hi, prob.bc)
        self.ctx.set_discretisation(prob.p, prob.gamma)
        self.ctx.set_penalty(prob.tau, prob.tau0)
        xv, _ = self.ctx.get_points(native.PTS_VOLUME, d)
        xi, _ = self.ctx.get_points(native.PTS_INTERIOR_FACE, d)
        xb, nb_ = self.ctx.get_points(native.PTS_BOUNDARY_FACE, d)
        self.points = (xv, xi, xb, nb_)
        self.ctx.set_viscosity(prob.mu(xv), prob.mu(xi) if len(xi) else np.zeros(0),
                               prob.mu(xb) if len(xb) else np.zeros(0))
        if prob.delta is not None:
            self.ctx.set_density(prob.rho(xv), prob.rho(xi) if len(xi) else np.zeros(0), prob.delta)
        self.chi = None
        if prob.phase is not None:
            centres = xv.reshape(prob.n_elements, -1, d).mean(axis=1)
            self.chi = np.asarray(prob.phase(centres), dtype=np.int32)
            self.ctx.set_phases(self.chi, prob.mu_phase, scale=prob.scale_mu)
        nu1, nu2 = (prob.nu1, prob.nu2) if nu is None else nu
        self.ctx.set_cycle(nu1, nu2, precision)
        if shape is not None:
            self.ctx.set_cycle_shape(*shape)
        self.ctx.set_colouring(colouring)
        self.ctx.set_clusters(clusters)
        self.ctx.set_bottom(bottom_max)
        if setup:
            self.ctx.setup()
            self.nlevels, self.ne_levels, self.nb, self.n_snapped = self.ctx.sizes()

    def rhs(self):
        """b from the manufactured solution of the problem (host array [ne][nb])."""
        prob, ex = self.prob, self.prob.exact
        d = prob.d
        xv, xi, xb, nrm = self.points
        f_vol = np.concatenate([ex.f(xv), ex.fdiv(xv)[:, None]], axis=1)
        bdata = np.zeros((len(xb), d))
        if len(xb):
            axis = np.argmax(np.abs(nrm), axis=1)
            side = np.sign(nrm[np.arange(len(xb)), axis]).astype(int)
            kind = np.array([prob.bc[2 * k + (0 if s < 0 else 1)] for k, s in zip(axis, side)])
            dmask = kind == DIRICHLET
            smask = kind == STRESS
            if dmask.any():
                bdata[dmask] = ex.u(xb[dmask])
            for k in range(d):
                for s in (-1, 1):
                    m = smask & (axis == k) & (side == s)
                    if m.any():
                        nvec = np.zeros(d)
                        nvec[k] = s
                        bdata[m] = ex.stress(xb[m], nvec)
        if self.chi is None:
            return self.ctx.assemble_rhs(f_vol, bdata, prob.n_elements, prob.nb)
        cm, cp, nrm_i = self.ctx.get_interface(len(xi), d)
        idata = np.zeros((len(xi), 2 * d))
        m = cm > 0
        if m.any():
            for k in range(d):
                for sg in (-1.0, 1.0):
                    sel = m & (nrm_i[:, k] == sg)
                    if sel.any():
                        nvec = np.zeros(d)
                        nvec[k] = sg
                        g, h = ex.jumps(xi[sel], nvec, cm[sel], cp[sel])
                        idata[sel, :d] = g
                        idata[sel, d:] = h
        return self.ctx.assemble_rhs2(f_vol, bdata, idata, prob.n_elements, prob.nb)

    def scaling(self):
        """Level-0 diagonal D of the sqrt(mu) scaling (ones without it)."""
        return self.ctx.get_scaling(self.prob.n_elements, self.prob.nb)

    def close(self):
        self.ctx.close()


class CutStokesMG:
    """The same for a problems.CutProblem: the embedded circle's cut-cell mesh
    (stk_set_levelset_circle), phase viscosities and densities, data sampled
    at the library's cut-cell points."""

    def __init__(self, prob, precision=native.FP64, device=0, nu=None, setup=True, bottom_max=0):
        self.prob = prob
        self.ctx = native.Context(device)
        self.ctx.set_mesh(2, (prob.n, prob.n), (0.0, 0.0), (1.0, 1.0), [DIRICHLET] * 4)
        self.ctx.set_discretisation(prob.p, prob.gamma)
        self.ctx.set_penalty(prob.tau, prob.tau0)
        self.ctx.set_levelset_circle(prob.centre, prob.radius)
        self.ctx.set_cut_phases(prob.mu_phase, scale=prob.scale_mu)
        if prob.unsteady:
            self.ctx.set_phase_density(prob.rho_phase, prob.delta)
        nu1, nu2 = (prob.nu1, prob.nu2) if nu is None else nu
        self.ctx.set_cycle(nu1, nu2, precision)
        self.ctx.set_bottom(bottom_max)
        if setup:
            self.ctx.setup()
            self.nlevels, self.ne_levels, self.nb, self.n_snapped = self.ctx.sizes()
            self.ne = int(self.ne_levels[0])

    def points(self, kind):
        x, n = self.ctx.get_points(kind, 2)
        return x, n, self.ctx.get_point_phases(kind)

    def rhs(self):
        """b of the manufactured two-phase problem (host array [ne][nb], unscaled)."""
        prob, ex = self.prob, self.prob.exact
        xv, _, cv = self.points(native.PTS_VOLUME)
        xb, _, cb = self.points(native.PTS_BOUNDARY_FACE)
        xi, ni, _ = self.points(native.PTS_INTERFACE)
        f_vol = prob.forcing(xv, cv)
        bdata = ex.u(xb, chi=cb)
        idata = np.zeros((len(xi), 4))
        if len(xi):
            one, two = np.ones(len(xi), dtype=int), np.full(len(xi), 2)
            idata[:, :2] = ex.u(xi, chi=one) - ex.u(xi, chi=two)
            # sigma n with the per-point normal: sigma e_0 n_0 + sigma e_1 n_1
            for k, ek in enumerate((np.array([1.0, 0.0]), np.array([0.0, 1.0]))):
                idata[:, 2:] += (ex.stress(xi, ek, chi=one) - ex.stress(xi, ek, chi=two)) * ni[:, k:k + 1]
        return self.ctx.assemble_rhs2(f_vol, bdata, idata, self.ne, self.nb)

    def scaling(self):
        return self.ctx.get_scaling(self.ne, self.nb)

    def close(self):
        self.ctx.close()
