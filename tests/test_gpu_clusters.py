"""Element clustering of the finest level (Concluding Remarks: larger
smoother blocks for p = 1) on the GPU against the oracle's cluster smoother.

With clusters of 2 x 2 elements the level-0 blocks are 48 x 48; the library
runs them on its element kernels in a cluster layout of the vectors.  FP64
V-cycle iterates must match the oracle's with the same clusters and colours
to 1e-12 (modulo the trivial kernel), solves must take the oracle's iteration
count (+-1), and a low-precision solve must need no more iterations than
without clusters.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1911_05888_gb300 import native, problems as P  # noqa: E402
from paper_1911_05888_gb300.solver import StokesMG  # noqa: E402
from oracle import multigrid  # noqa: E402

pytestmark = pytest.mark.gpu

# V(3,3), the paper's cycle: with V(1,1) plain iterative refinement does not
# contract on the periodic p = 1 problem (the oracle's diverges as well, with or
# without clusters), although GMRES preconditioned by the same cycle does.
CASES = {
    "vs-dirichlet-stress-p1": lambda: P.generic(2, 16, 1, 1, [P.DIRICHLET] * 3 + [P.STRESS],
                                                exact=P.paper_solution(2, 1), nu=(3, 3)),
    "std-periodic-p1": lambda: P.generic(2, 16, 1, 0, [P.PERIODIC] * 4, exact=P.paper_solution(2, 0), nu=(3, 3)),
    "std-rect-p1": lambda: P.generic(2, (12, 8), 1, 0, [P.DIRICHLET, P.STRESS, P.DIRICHLET, P.DIRICHLET],
                                     exact=P.paper_solution(2, 0), nu=(3, 3)),
}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def kernel_basis(prob, orc):
    lev = orc.levels[0]
    cols = []
    for v in range(prob.d + 1):
        z = np.zeros((lev.ne, lev.nb))
        z[:, v * lev.s] = 1.0
        z = z.ravel()
        if np.linalg.norm(lev.A @ z) <= 1e-10 * abs(lev.A).max() * np.linalg.norm(z):
            cols.append(z)
    if not cols:
        return np.zeros((prob.n_dofs, 0))
    return np.linalg.qr(np.stack(cols, axis=1))[0]


@pytest.mark.parametrize("name", list(CASES))
def test_clustered_cycle_matches_oracle(name):
    prob = CASES[name]()
    gpu = StokesMG(prob, clusters=True)
    orc = multigrid.Multigrid(prob, two_colours=prob.gamma == 0, clusters=True)
    try:
        assert gpu.ctx.info(native.INFO_CLUSTERS) == 1 and orc.clusters
        Z = kernel_basis(prob, orc)
        b = np.random.default_rng(21).uniform(-1, 1, prob.n_dofs)
        b -= Z @ (Z.T @ b)
        xd = torch.zeros(prob.n_dofs, dtype=torch.float64, device="cuda")
        xo = np.zeros(prob.n_dofs)
        for k in range(10):
            gpu.ctx.vcycle(xd, dev(b))
            orc.vcycle(xo, b)
            xg = xd.cpu().numpy()
            assert rel(xg - Z @ (Z.T @ xg), xo - Z @ (Z.T @ xo)) <= 1e-12, k
        bs = gpu.rhs().ravel()
        x = torch.zeros(prob.n_dofs, dtype=torch.float64, device="cuda")
        it, hist = gpu.ctx.solve(x, dev(bs), rtol=1e-10, maxit=100)
        xs, hs = orc.solve(bs, rtol=1e-10, maxit=100)
        assert hist[-1] <= 1e-10 and abs(it - (len(hs) - 1)) <= 1
        assert rel(x.cpu().numpy(), xs) <= 1e-10
    finally:
        gpu.close()


@pytest.mark.parametrize("precision", [native.FP32, native.FP16])
def test_clustered_low_precision_solve_needs_no_more_iterations(precision):
    prob = CASES["vs-dirichlet-stress-p1"]().with_(n=(32, 32))
    its = {}
    for on in (False, True):
        gpu = StokesMG(prob, precision=precision, clusters=on)
        try:
            assert gpu.ctx.info(native.INFO_CLUSTERS) == int(on)
            gpu.ctx.set_solver(native.FGMRES, 30)
            b = dev(gpu.rhs().ravel())
            x = torch.zeros_like(b)
            its[on], hist = gpu.ctx.solve(x, b, rtol=1e-10, maxit=100)
            assert hist[-1] <= 1e-10
        finally:
            gpu.close()
    assert its[True] <= its[False], its


def test_clusters_only_where_they_apply():
    """A periodic axis with 3 clusters (n = 6), a degree above 1, or a 3D mesh
    keeps element blocks."""
    for prob in (P.generic(2, 12, 1, 1, [P.PERIODIC] * 4).with_(n=(6, 12)),
                 P.generic(2, 8, 2, 1, [P.DIRICHLET] * 4),
                 P.generic(3, 4, 1, 0, [P.DIRICHLET] * 6)):
        gpu = StokesMG(prob, clusters=True)
        try:
            assert gpu.ctx.info(native.INFO_CLUSTERS) == 0
        finally:
            gpu.close()
