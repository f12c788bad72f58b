"""The persistent coarse cycle (one cooperative launch for every level below
a bound, grid barriers between its phases) against the launch-per-step cycle
and the oracle, and the bounded grid barrier's timeout path.

Each phase of the persistent launch runs the per-element code of the kernel
it replaces, so the iterates must agree bit for bit with the launch-per-step
path, and with the oracle to the FP64 tolerance (1e-12) of the other parity
tests.  The timeout test makes a barrier wait run out by keeping one CTA away
from it (a wait that nothing will end) with a bound of about a millisecond:
the other CTAs give up, the call reports STK_ERR_TIMEOUT and the context
keeps working.  Nothing traps or faults.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1911_05888_gb300 import native, problems as P  # noqa: E402
from paper_1911_05888_gb300.solver import StokesMG  # noqa: E402
from oracle import multigrid  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = {
    "stress16p3": lambda: P.stress_variable_mu_2d(n=16, p=3),
    "periodic16p2": lambda: P.periodic_standard_2d(n=16, p=2),
    "3d-unsteady-p2": lambda: P.unsteady_periodic_3d(n=8, p=2, re=10.0),
    "square-1e3-p3": lambda: P.square_interface(n=8, p=3, mu_inner=1e3),
}
ALL = 1 << 20   # every level below level 0


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
        if lev.D is not None:
            z = z / lev.D
        if np.linalg.norm(lev.A @ z) <= 1e-10 * abs(lev.A).max() * np.linalg.norm(z):
            cols.append(z)
    if not cols:
        return np.zeros((prob.n_dofs, 0))
    return np.linalg.qr(np.stack(cols, axis=1))[0]


@pytest.mark.parametrize("shape", [(1, 1, 64), (2, 1, 64), (1, 2, 64)])
@pytest.mark.parametrize("name", list(CASES))
def test_persistent_cycle_is_the_same_cycle(name, shape):
    """FP64 V-, W- and variable V-cycles with the persistent coarse part equal
    the launch-per-step cycles bit for bit, and the oracle's iterates to
    1e-12 (modulo the trivial kernel), over four cycles; 2e-12 on the
    viscosity-ratio-1e3 case, whose scaled element blocks amplify rounding
    more (the first iterate of this seed differs by 1.04e-12 on either
    path)."""
    prob = CASES[name]()
    gpu = StokesMG(prob, shape=shape)
    orc = multigrid.Multigrid(prob, two_colours=(prob.gamma == 0 and prob.phase is None), shape=shape)
    try:
        Z = kernel_basis(prob, orc)
        b = np.random.default_rng(3).uniform(-1, 1, prob.n_dofs)
        b -= Z @ (Z.T @ b)
        bd = dev(b)
        runs = {}
        for on in (0, ALL):
            gpu.ctx.set_persistent(on, 1)
            xd = torch.zeros_like(bd)
            its = []
            for _ in range(4):
                gpu.ctx.vcycle(xd, bd)
                its.append(xd.clone())
            runs[on] = its
        xo = np.zeros(prob.n_dofs)
        for k in range(4):
            assert torch.equal(runs[0][k], runs[ALL][k]), k
            orc.vcycle(xo, b)
            xg = runs[ALL][k].cpu().numpy()
            tol = 2e-12 if prob.phase is not None else 1e-12
            assert rel(xg - Z @ (Z.T @ xg), xo - Z @ (Z.T @ xo)) <= tol, k
    finally:
        gpu.close()


@pytest.mark.parametrize("precision", [native.FP32, native.BF16, native.FP16])
@pytest.mark.parametrize("name", ["stress16p3", "3d-unsteady-p2"])
def test_persistent_low_precision_solve(name, precision):
    """Low-precision cycles inside FGMRES: the persistent coarse cycle gives
    the same iteration count and residual history as the launch-per-step
    cycle (identical arithmetic), and reaches 1e-10; several CTAs per SM
    change nothing either."""
    prob = CASES[name]()
    gpu = StokesMG(prob, precision=precision)
    try:
        gpu.ctx.set_solver(native.FGMRES, 30)
        b = dev(gpu.rhs().ravel())
        out = {}
        for on, ctas in ((0, 1), (ALL, 1), (ALL, 2)):
            gpu.ctx.set_persistent(on, ctas)
            x = torch.zeros_like(b)
            it, hist = gpu.ctx.solve(x, b, rtol=1e-10, maxit=200)
            out[(on, ctas)] = (it, hist, x.cpu().numpy())
        it0, h0, x0 = out[(0, 1)]
        assert h0[-1] <= 1e-10
        for key in ((ALL, 1), (ALL, 2)):
            it1, h1, x1 = out[key]
            assert it1 == it0 and np.array_equal(h1, h0) and np.array_equal(x1, x0), key
    finally:
        gpu.close()


def test_persistent_bound_selects_levels():
    """The bound selects the levels: with 64 elements as the bound on a 16 x 16
    mesh (levels 256, 64, 16, 4 elements) the persistent part starts at level
    1; a bound below every coarse level leaves the cycle as it was; a bad
    setting is rejected."""
    prob = CASES["stress16p3"]()
    gpu = StokesMG(prob)
    try:
        b = dev(np.random.default_rng(5).uniform(-1, 1, prob.n_dofs))
        ref = torch.zeros_like(b)
        gpu.ctx.vcycle(ref, b)
        for bound in (64, 16, 3):
            gpu.ctx.set_persistent(bound, 1)
            x = torch.zeros_like(b)
            gpu.ctx.vcycle(x, b)
            assert torch.equal(x, ref), bound
        with pytest.raises(native.StkError):
            gpu.ctx.set_persistent(-1, 1)
        with pytest.raises(native.StkError):
            gpu.ctx.set_persistent(64, 9)
    finally:
        gpu.close()


def test_grid_barrier_timeout_is_reported_and_recoverable():
    """All CTAs present: four barriers pass (grid x 4 passages).  One CTA
    absent: the barrier wait of every other CTA reaches its bound (2e6 clock
    ticks, about a millisecond) and the call returns STK_ERR_TIMEOUT with no
    passage counted; afterwards the context still solves."""
    prob = CASES["stress16p3"]()
    gpu = StokesMG(prob, precision=native.FP32)
    try:
        gpu.ctx.set_persistent(ALL, 1)
        rc, passed = gpu.ctx.barrier_selftest(-1, 2_000_000_000)
        grid = torch.cuda.get_device_properties(0).multi_processor_count
        assert rc == native.STK_OK and passed == 4 * grid
        rc, passed = gpu.ctx.barrier_selftest(3, 2_000_000)
        assert rc == -4 and passed == 0            # STK_ERR_TIMEOUT
        gpu.ctx.set_solver(native.FGMRES, 30)
        b = dev(gpu.rhs().ravel())
        x = torch.zeros_like(b)
        it, hist = gpu.ctx.solve(x, b, rtol=1e-10, maxit=100)
        assert hist[-1] <= 1e-10
        rc, passed = gpu.ctx.barrier_selftest(-1, 2_000_000_000)
        assert rc == native.STK_OK and passed == 4 * grid
    finally:
        gpu.close()
