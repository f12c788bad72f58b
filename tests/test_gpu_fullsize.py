"""Full-size checks on the workload the benchmark times: 2D viscous-stress
form, 256 x 256 elements, p = 3, Dirichlet on three sides and a stress
condition on the fourth, mu = 1 + 0.9 sin(2 pi x) cos(2 pi y), V(3,3) cycles
with FP32-stored blocks inside FP64 flexible GMRES.  The finest-level colour
steps run in the same launch configuration as in the benchmark (one warp per
element; 16384 elements per launch).

The oracle cannot assemble this mesh in seconds, so the checks are
(1) sampled outputs recomputed one element at a time from the block
definition of the colour step and the residual (Section 3; Algorithm 1),
using the library's own FP64 blocks -- which equal the oracle's to 1e-13 on
every small case of test_gpu_parity -- and bounded by the rounding-error
bound of the arithmetic: a dot product of n terms computed in unit
roundoff u is off by at most gamma_n = n u / (1 - n u) times the sum of the
absolute values of its terms; and
(2) properties of the solve that hold at any size: every sampled element's
FP64 residual, recomputed in numpy, is below the solve's 1e-10 bound, and
the velocity and pressure errors against the manufactured solution are
below those of the oracle's 64 x 64 solve divided by the convergence factor
the oracle shows (order p+1 for u, about p+1/2 for p; Appendix C).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1911_05888_gb300 import native, problems as P  # noqa: E402
from paper_1911_05888_gb300.solver import StokesMG  # noqa: E402
from oracle import basis, ldg, multigrid  # noqa: E402

pytestmark = pytest.mark.gpu

N, DEG = 256, 3
U32, U64 = 2.0 ** -24, 2.0 ** -53

_cache = {}


def problem():
    return P.stress_variable_mu_2d(n=N, p=DEG, nu=(3, 3))


def solver(precision):
    if precision not in _cache:
        _cache[precision] = StokesMG(problem(), precision=precision)
    return _cache[precision]


def gamma(n, u):
    return n * u / (1 - n * u)


def neighbours(i):
    """Natural indices of the elements within one step along each axis
    (the reach of the viscous-stress couplings), inside the box."""
    ix, iy = i % N, i // N
    out = []
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            jx, jy = ix + dx, iy + dy
            if (dx or dy) and 0 <= jx < N and 0 <= jy < N:
                out.append(jy * N + jx)
    return out


def sampled_colour0(rng, k):
    """k random elements of parity colour 0 (both indices even)."""
    ix = 2 * rng.integers(0, N // 2, k)
    iy = 2 * rng.integers(0, N // 2, k)
    return np.unique(iy * N + ix)


def element_terms(gpu, i, x, b):
    """A_ii, A_ii^{-1} and g_i = b_i - sum_j A_ij x_j with the term sums
    sum |b| + sum_j |A_ij| |x_j| (FP64 numpy, blocks from the library)."""
    nb = gpu.nb
    g = b[i].copy()
    mag = np.abs(b[i]).copy()
    nterms = 1
    for j in neighbours(i):
        A = gpu.ctx.get_block(0, int(i), int(j), nb)
        if not A.any():
            continue
        g -= A @ x[j]
        mag += np.abs(A) @ np.abs(x[j])
        nterms += nb
    Aii = gpu.ctx.get_block(0, int(i), int(i), nb)
    return Aii, g, mag, nterms


def round_subblocks16(A, s):
    """FP16 with one power-of-two scale per s x s sub-block (the library's
    coupling records), via the oracle's rounding."""
    nb = A.shape[0]
    q = nb // s
    B = A.reshape(q, s, q, s).transpose(0, 2, 1, 3)
    return multigrid.round_fp16_scaled(B, axis=(2, 3)).transpose(0, 2, 1, 3).reshape(nb, nb)


@pytest.mark.parametrize("precision", [native.FP64, native.FP32, native.FP16])
def test_fullsize_colour_step_sampled(precision):
    """One finest-level colour step at full size, sampled elements.
    FP32 / FP16 blocks: against x_i = A_ii^{-1} (b_i - sum_j A_ij x_j)
    evaluated in FP64 on the same FP32-rounded inputs and the same rounded
    blocks, within gamma_n of FP32 arithmetic (plus one unit in the last place
    of each rounded inverse entry, as the library's and numpy's FP64 inverses
    round independently).  FP64 blocks: the new x_i solves A_ii x_i = g_i to
    a backward error of 1e-12."""
    gpu = solver(precision)
    nb = gpu.nb
    rng = np.random.default_rng(7)
    x0 = rng.uniform(-1, 1, (N * N, nb))
    b = rng.uniform(-1, 1, (N * N, nb))
    fp32 = precision != native.FP64
    if fp32:
        x0 = x0.astype(np.float32).astype(np.float64)
        b = b.astype(np.float32).astype(np.float64)
    dt = torch.float32 if fp32 else torch.float64
    xd = torch.from_numpy(x0.ravel()).to(dt).cuda()
    bd = torch.from_numpy(b.ravel()).to(dt).cuda()
    gpu.ctx.gs_colour_ex(0, 0, precision, xd, bd)
    torch.cuda.synchronize()
    xg = xd.double().cpu().numpy().reshape(N * N, nb)
    if precision == native.FP32:
        rnd = rnd_inv = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
        u_inv = U32
    elif precision == native.FP16:
        s = (DEG + 1) ** 2
        rnd = lambda a: round_subblocks16(a, s)  # noqa: E731
        rnd_inv = lambda a: multigrid.round_fp16_scaled(a, axis=1)  # noqa: E731
        u_inv = 2.0 ** -11
    else:
        rnd = rnd_inv = lambda a: a  # noqa: E731
    for i in sampled_colour0(rng, 48):
        g = b[i].copy()
        mag = np.abs(b[i]).copy()
        nterms = 1
        for j in neighbours(i):
            A = rnd(gpu.ctx.get_block(0, int(i), int(j), nb))
            if A.any():
                g -= A @ x0[j]
                mag += np.abs(A) @ np.abs(x0[j])
                nterms += nb
        Aii = gpu.ctx.get_block(0, int(i), int(i), nb)
        if fp32:
            Ainv = rnd_inv(np.linalg.inv(Aii))
            ref = Ainv @ g
            gn = gamma(nterms + 8, U32) * mag
            bound = (np.abs(Ainv) @ gn + (gamma(nb + 1, U32) + 2 * u_inv) * (np.abs(Ainv) @ (np.abs(g) + gn))
                     + U32 * np.abs(ref))
            err = np.abs(xg[i] - ref)
            assert np.all(err <= bound), (i, err.max(), bound.max(), np.linalg.cond(Aii))
        else:
            res = Aii @ xg[i] - g
            scale = np.abs(Aii) @ np.abs(xg[i]) + mag
            assert np.all(np.abs(res) <= 1e-12 * scale), (i, np.abs(res / scale).max())
    # elements of the other colours are untouched
    e = np.arange(N * N)
    other = np.nonzero(((e % N) % 2) | ((e // N) % 2))[0]
    assert np.array_equal(xg[other], x0[other])


def test_fullsize_fp64_residual_sampled():
    """The FP64 outer residual r = b - A x at full size: sampled elements
    against the block definition, within gamma_n in FP64."""
    gpu = solver(native.FP64)
    nb = gpu.nb
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, (N * N, nb))
    b = rng.uniform(-1, 1, (N * N, nb))
    xd = torch.from_numpy(x.ravel()).cuda()
    bd = torch.from_numpy(b.ravel()).cuda()
    r = torch.empty_like(xd)
    gpu.ctx.residual(xd, bd, r)
    rg = r.cpu().numpy().reshape(N * N, nb)
    for i in rng.choice(N * N, 64, replace=False):
        Aii, g, mag, nterms = element_terms(gpu, i, x, b)
        ref = g - Aii @ x[i]
        mag = mag + np.abs(Aii) @ np.abs(x[i])
        assert np.all(np.abs(rg[i] - ref) <= gamma(nterms + nb, U64) * mag), i


def l2_errors(prob, x):
    """L2 errors of u (per component) and p against the manufactured
    solution, from the coefficients x[element][variable][mode]."""
    mesh = ldg.Mesh(prob.d, prob.n, prob.lo, prob.hi, prob.bc)
    q = prob.p + 3
    xv, wv = mesh.volume_points(q)
    Phi = basis.tensor_basis(prob.d, prob.p, q)
    s = (prob.p + 1) ** prob.d
    vals = np.einsum("qa,eva->eqv", Phi, x.reshape(mesh.ne, prob.d + 1, s))
    ue, pe = prob.exact.u(xv), prob.exact.p(xv)
    jac = mesh.vol / 2 ** prob.d
    out = []
    for v in range(prob.d + 1):
        err = vals[..., v] - (ue[..., v] if v < prob.d else pe)
        out.append(np.sqrt(jac * (err ** 2 * wv).sum()))
    return np.array(out)


def test_fullsize_solve_residual_and_accuracy():
    """The benchmark's solve (FP32 V(3,3) in FP64 flexible GMRES) at full
    size: 1e-10 relative residual, confirmed element by element in numpy,
    and discretisation errors at the oracle's convergence orders."""
    prob = problem()
    gpu = solver(native.FP32)
    gpu.ctx.set_solver(native.FGMRES, 30)
    b = gpu.rhs()
    bd = torch.from_numpy(b.ravel()).cuda()
    xd = torch.zeros_like(bd)
    try:
        it, hist = gpu.ctx.solve(xd, bd, rtol=1e-10, maxit=60)
        assert hist[-1] <= 1e-10 and it <= 15, (it, hist)
        x = xd.cpu().numpy().reshape(N * N, -1)
        # continue from x to 1e-13 so that the discretisation error, not the
        # algebraic one, is what the accuracy check below sees
        it2, hist2 = gpu.ctx.solve(xd, bd, rtol=1e-13, maxit=60)
        assert hist2[-1] <= 1e-13, hist2
    finally:
        gpu.ctx.set_solver(native.RICHARDSON, 30)
    gpu64 = solver(native.FP64)
    rng = np.random.default_rng(4)
    bn = np.linalg.norm(b)
    edge = [0, N - 1, N * (N - 1), N * N - 1, N // 2, N * (N // 2)]
    for i in list(rng.choice(N * N, 48, replace=False)) + edge:
        Aii, g, _, _ = element_terms(gpu64, i, x, b)
        assert np.linalg.norm(g - Aii @ x[i]) <= 1e-10 * bn, i
    x = xd.cpu().numpy().reshape(N * N, -1)
    # Oracle at 64 x 64 (order p+1 for u, about p+1/2 for p, Appendix C):
    # two halvings of h must gain at least order p+1/2 for u and p for p.
    small = P.stress_variable_mu_2d(n=64, p=DEG, nu=(3, 3))
    mg = multigrid.Multigrid(small)
    bo = mg.levels[0].P @ ldg.rhs(small, mg.levels[0].ops)
    xo, ho = mg.solve(bo, rtol=1e-12, maxit=300)
    e64 = l2_errors(small, xo)
    e256 = l2_errors(prob, x)
    assert np.all(e256[:2] <= e64[:2] / 4.0 ** (DEG + 0.5)), (e256, e64)
    assert e256[2] <= e64[2] / 4.0 ** DEG, (e256, e64)
