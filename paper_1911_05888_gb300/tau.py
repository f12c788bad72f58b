"""Pressure-penalty sweep of Section 4 on the GPU.

The convergence rate rho of eq. (rho) -- average reduction per iteration of
V-cycle left-preconditioned GMRES on V A x = 0 from a random (d+1)-field x0,
run until the residual falls by 1e-8 -- is evaluated over a log-spaced grid
of tau (eq. taueqn's prefactor).  From the grid come the minimiser (the
quantity of Table 1) and the window of tau whose rho is at most
(min rho)^(1 - eps), eps = 1/9, i.e. at most 12.5 % more iterations than at
the minimum (Table 2).  Every rho is computed by the library's
``stk_gmres_rho``; this module only picks tau values, builds contexts and
reads the results.

Command line: ``python -m paper_1911_05888_gb300.tau --cases 0,2,2 1,2,3
--n 128`` prints one JSON line per (form, d, p) case.  ``--disc 32 64 128
--disc-p 2 3`` instead prints rho on Section 5's curved domain (the disc of
radius 0.45 on an n x n background grid, standard form, mu = 1, Dirichlet data
on the circle) with Table 1's tau; ``--bubble 32 64 128`` the same for the
water / gas bubble of Section 6.
"""
import argparse
import json
import math
import time

import numpy as np

from . import native, problems as P
from .solver import StokesMG

EPS = 1.0 / 9.0


def rho_of(prob, tau, precision=native.FP64, seed=1, reduction=1e-8, maxit=100, shape=None):
    """(rho, iterations) of eq. (rho) for prob with the penalty prefactor tau."""
    import torch
    q = prob.with_(tau=tau)
    mg = StokesMG(q, precision=precision, shape=shape)
    try:
        x0 = torch.from_numpy(P.random_vector(q.n_elements, q.nb, seed=seed).ravel()).cuda()
        r, n, _, _ = mg.ctx.gmres_rho(x0, reduction, maxit)
    finally:
        mg.ctx.close()
    return r, n


def disc_rho(n, p, precision=native.FP64, seed=1, reduction=1e-8, maxit=100):
    """(rho, iterations, elements) of eq. (rho) on the disc of radius 0.45 cut
    from an n x n grid (standard form, mu = 1, Table 1's tau)."""
    import torch
    from .solver import CutStokesMG
    prob = P.CutProblem(n=n, p=p, gamma=0, mu_phase=(1.0,), radius=0.45, inside_only=True)
    mg = CutStokesMG(prob, precision=precision)
    try:
        x0 = torch.from_numpy(P.random_vector(mg.ne, mg.nb, seed=seed).ravel()).cuda()
        r, it, _, _ = mg.ctx.gmres_rho(x0, reduction, maxit)
    finally:
        mg.close()
    return r, it, mg.ne


def bubble_rho(n, p, water_inside, precision=native.FP64, seed=1, reduction=1e-8, maxit=100, bottom_max=0):
    """(rho, iterations, elements) of eq. (rho) for the paper's time-dependent
    two-phase bubble (Section 6): the circle of radius 0.3 in the unit
    square, water (rho = 1, mu = 1) and gas (rho = 1e-3, mu = 2e-4), delta =
    0.1 h, viscous-stress form, Dirichlet box, sqrt(mu) scaling; water inside
    (water_inside) or gas inside."""
    import torch
    from .solver import CutStokesMG
    water, gas = (1.0, 1.0), (1e-3, 2e-4)   # (rho, mu)
    inside, outside = (water, gas) if water_inside else (gas, water)
    prob = P.CutProblem(n=n, p=p, gamma=1, mu_phase=(inside[1], outside[1]), rho_phase=(inside[0], outside[0]),
                        delta=0.1 / n, radius=0.3)
    mg = CutStokesMG(prob, precision=precision, bottom_max=bottom_max)
    try:
        x0 = torch.from_numpy(P.random_vector(mg.ne, mg.nb, seed=seed).ravel()).cuda()
        r, it, _, _ = mg.ctx.gmres_rho(x0, reduction, maxit)
    finally:
        mg.close()
    return r, it, mg.ne


def parabolic_min(t, r):
    """Vertex of the parabola through three (log tau, log rho) points around
    the grid minimum (the grid point itself when the minimum is on the edge)."""
    k = int(np.argmin(r))
    if k == 0 or k == len(r) - 1:
        return t[k]
    x = np.log(t[k - 1:k + 2])
    y = np.log(r[k - 1:k + 2])
    den = (x[0] - x[1]) * (x[0] - x[2]) * (x[1] - x[2])
    a = (x[2] * (y[1] - y[0]) + x[1] * (y[0] - y[2]) + x[0] * (y[2] - y[1])) / den
    b = (x[2] ** 2 * (y[0] - y[1]) + x[1] ** 2 * (y[2] - y[0]) + x[0] ** 2 * (y[1] - y[2])) / den
    if a <= 0:
        return t[k]
    return float(np.exp(-b / (2 * a)))


def window(t, r, eps=EPS):
    """Ends of the connected range of tau around the grid minimum with
    rho <= (min rho)^(1 - eps), interpolated linearly in (log tau, log rho)
    between grid points; None for an end that lies outside the grid."""
    k = int(np.argmin(r))
    thr = math.log(r[k]) * (1.0 - eps)
    lr = np.log(np.asarray(r))
    lt = np.log(np.asarray(t))
    ends = []
    for step in (-1, 1):
        j = k
        while 0 <= j + step < len(r) and lr[j + step] <= thr:
            j += step
        if not 0 <= j + step < len(r):
            ends.append(None)
            continue
        f = (thr - lr[j]) / (lr[j + step] - lr[j])
        ends.append(float(np.exp(lt[j] + f * (lt[j + step] - lt[j]))))
    return tuple(ends)


def sweep(form, d, p, n, per_octave=4, octaves=2, centre=None, precision=native.FP64, nu=(3, 3)):
    """rho over tau = centre * 2^(k / per_octave), |k| <= octaves * per_octave,
    on the periodic unit square / cube with mu = 1 (Section 4's setting)."""
    centre = P.TABLE1_TAU[(form, d, p)] if centre is None else centre
    prob = P.generic(d, n, p, form, [P.PERIODIC] * (2 * d), nu=nu)
    ks = range(-octaves * per_octave, octaves * per_octave + 1)
    taus = [centre * 2.0 ** (k / per_octave) for k in ks]
    rhos, its = [], []
    for t in taus:
        r, it = rho_of(prob, t, precision=precision)
        rhos.append(r)
        its.append(it)
    return np.array(taus), np.array(rhos), np.array(its)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--cases", nargs="+", default=["0,2,2"], help="form,d,p (form 0 standard, 1 viscous stress)")
    ap.add_argument("--n", type=int, default=128, help="elements per axis (2D)")
    ap.add_argument("--n3", type=int, default=32, help="elements per axis (3D)")
    ap.add_argument("--per-octave", type=int, default=4)
    ap.add_argument("--octaves", type=int, default=2)
    ap.add_argument("--disc", type=int, nargs="*", default=None, help="background grid sizes of the disc")
    ap.add_argument("--disc-p", type=int, nargs="+", default=[2, 3])
    ap.add_argument("--bubble", type=int, nargs="*", default=None,
                    help="background grid sizes of the water / gas bubble (Section 6)")
    args = ap.parse_args(argv)
    if args.bubble:
        for water_inside in (True, False):
            for p in args.disc_p:
                for n in args.bubble:
                    t0 = time.perf_counter()
                    r, it, ne = bubble_rho(n, p, water_inside)
                    print(json.dumps({"problem": "water bubble in gas" if water_inside else "gas bubble in water",
                                      "radius": 0.3, "delta": "0.1 h", "p": p, "n": n, "elements": ne,
                                      "tau": P.TABLE1_TAU[(1, 2, p)], "rho": round(r, 4), "iterations": it,
                                      "seconds": round(time.perf_counter() - t0, 1)}), flush=True)
        return
    if args.disc:
        for p in args.disc_p:
            for n in args.disc:
                t0 = time.perf_counter()
                r, it, ne = disc_rho(n, p)
                print(json.dumps({"domain": "disc r = 0.45, standard form, mu = 1, Dirichlet", "p": p, "n": n,
                                  "elements": ne, "tau": P.TABLE1_TAU[(0, 2, p)], "rho": round(r, 4),
                                  "iterations": it, "seconds": round(time.perf_counter() - t0, 1)}), flush=True)
        return
    for case in args.cases:
        form, d, p = (int(v) for v in case.split(","))
        n = args.n if d == 2 else args.n3
        t0 = time.perf_counter()
        taus, rhos, its = sweep(form, d, p, n, args.per_octave, args.octaves)
        k = int(np.argmin(rhos))
        lo, hi = window(taus, rhos)
        print(json.dumps({
            "form": ["standard", "viscous-stress"][form], "d": d, "p": p, "n": n,
            "table1_tau": P.TABLE1_TAU[(form, d, p)], "table2_window": P.TABLE2_WINDOW[(form, d, p)],
            "argmin_grid": taus[k], "argmin_parabolic": parabolic_min(taus, rhos), "min_rho": rhos[k],
            "window": [lo, hi], "rho_at_table1": rhos[len(rhos) // 2],
            "tau": [float("%.5g" % t) for t in taus], "rho": [float("%.4f" % r) for r in rhos],
            "iterations": [int(i) for i in its], "seconds": round(time.perf_counter() - t0, 1)}), flush=True)


if __name__ == "__main__":
    main()
