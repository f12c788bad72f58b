"""A batch of independent problems solved in one persistent launch
(stk_solve_batch_persistent) against the oracle and against the library's
own one-problem solves.

The batch mixes mesh sizes (8^2 .. 16^2, one with an odd 3 x 3 bottom),
degrees (p = 2, 3) and seeded viscosity contrasts of the 2D unsteady
viscous-stress serving workload.  Every problem must reach 1e-10 with the
iteration count of the oracle's iterative refinement with the same FP32
rounding of the blocks (+-1), give the oracle's solution to 1e-8 and satisfy
||b - A x|| <= 1e-10 ||b|| with the oracle's FP64 operator.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1911_05888_gb300 import native, problems as P  # noqa: E402
from paper_1911_05888_gb300.solver import StokesMG  # noqa: E402
from oracle import multigrid  # noqa: E402

pytestmark = pytest.mark.gpu

MIX = [(8, 2, 0), (16, 3, 1), (12, 2, 2), (8, 3, 4)]


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def test_persistent_batch_matches_oracle_and_single_solves():
    probs = [P.unsteady_stress_2d(n=n, p=p, seed=seed) for n, p, seed in MIX]
    gpus = [StokesMG(q, precision=native.FP32) for q in probs]
    try:
        bh = [g.rhs().ravel() for g in gpus]
        bs = [torch.from_numpy(b).cuda() for b in bh]
        xs = [torch.zeros_like(b) for b in bs]
        its, status, hist = native.solve_batch_persistent([g.ctx for g in gpus], xs, bs, rtol=1e-10, maxit=100)
        assert status == [native.STK_OK] * len(gpus)
        for q, g, b, x, it, h in zip(probs, gpus, bh, xs, its, hist):
            assert 0 < it < 100 and h[it] <= 1e-10 and np.all(h[it + 1:] == 0), (it, h[: it + 1])
            xg = x.cpu().numpy()
            orc = multigrid.Multigrid(q, storage="fp32")
            xo, ho = orc.solve(b, rtol=1e-10, maxit=100)
            assert abs(it - (len(ho) - 1)) <= 1, (it, len(ho) - 1)
            assert rel(xg, xo) <= 1e-8
            assert np.linalg.norm(b - orc.A @ xg) <= 1e-10 * np.linalg.norm(b)
            # the library's one-problem iterative refinement with the same cycle
            g.ctx.set_solver(native.RICHARDSON, 30)
            x1 = torch.zeros_like(x)
            it1, h1 = g.ctx.solve(x1, torch.from_numpy(b).cuda(), rtol=1e-10, maxit=100)
            assert abs(it1 - it) <= 1 and rel(xg, x1.cpu().numpy()) <= 1e-8
        # a second call on the same contexts from a non-zero start converges at once
        its2, status2, hist2 = native.solve_batch_persistent([g.ctx for g in gpus], xs, bs, rtol=1e-9, maxit=100)
        assert status2 == [native.STK_OK] * len(gpus) and its2 == [0] * len(gpus)
    finally:
        for g in gpus:
            g.close()


def test_persistent_batch_refuses_what_it_cannot_run():
    """FP64 contexts, a context twice, and a context that is not set up are
    refused before any launch."""
    a = StokesMG(P.unsteady_stress_2d(n=8, p=2, seed=0), precision=native.FP32)
    f64 = StokesMG(P.unsteady_stress_2d(n=8, p=2, seed=1), precision=native.FP64)
    try:
        b = torch.from_numpy(a.rhs().ravel()).cuda()
        x = torch.zeros_like(b)
        with pytest.raises(native.StkError):
            native.solve_batch_persistent([a.ctx, f64.ctx], [x, x.clone()], [b, b.clone()])
        with pytest.raises(native.StkError):
            native.solve_batch_persistent([a.ctx, a.ctx], [x, x.clone()], [b, b.clone()])
    finally:
        a.close()
        f64.close()
