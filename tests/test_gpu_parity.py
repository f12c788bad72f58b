"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

FP64 tolerances: operator blocks 1e-13 (relative to the level's largest
entry), single kernels 1e-13, V-cycle iterates 1e-12 relative (the stated
target).  Low-precision cycles are judged by the FP64 outer iteration
reaching 1e-10 and by their distance to the oracle's emulation of the same
rounding.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1911_05888_gb300 import native, problems as P  # noqa: E402
from paper_1911_05888_gb300.solver import StokesMG  # noqa: E402
from oracle import multigrid  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = {
    "periodic16p2": lambda: P.periodic_standard_2d(n=16, p=2),
    "stress16p3": lambda: P.stress_variable_mu_2d(n=16, p=3),
    "dirichlet-rect": lambda: P.generic(2, (12, 8), 2, 0, [P.DIRICHLET, P.STRESS, P.DIRICHLET, P.DIRICHLET],
                                        exact=P.paper_solution(2, 0)),
    "vs-periodic-p1": lambda: P.generic(2, 8, 1, 1, [P.PERIODIC] * 4, exact=P.paper_solution(2, 1)),
    "3d-mixed-p1": lambda: P.generic(3, 4, 1, 1, [P.DIRICHLET, P.STRESS, P.PERIODIC, P.PERIODIC,
                                                  P.DIRICHLET, P.DIRICHLET], exact=P.paper_solution(3, 1)),
    "3d-unsteady-p2": lambda: P.unsteady_periodic_3d(n=8, p=2, re=10.0),
    "square-1e-3": lambda: P.square_interface(n=16, p=2, mu_inner=1e-3),
    "square-1e3-p3": lambda: P.square_interface(n=8, p=3, mu_inner=1e3),
    # 6^3 -> 3^3: a 2916-unknown bottom level, the size that takes the
    # equilibrated cuSOLVER eigensolver (3D unsteady workloads of 48^3 end there)
    "3d-unsteady-6p2": lambda: P.unsteady_periodic_3d(n=6, p=2, re=10.0),
}

_cache = {}


def oracle_for(prob, **kw):
    """The oracle with the library's default colouring: the checkerboard for
    the single-phase standard form, the 2^d parity colours otherwise."""
    return multigrid.Multigrid(prob, two_colours=(prob.gamma == 0 and prob.phase is None), **kw)


def get(name, precision=native.FP64):
    key = (name, precision)
    if key not in _cache:
        prob = CASES[name]()
        gpu = StokesMG(prob, precision=precision)
        orc = oracle_for(prob) if (name, native.FP64) not in _cache else _cache[(name, native.FP64)][2]
        _cache[key] = (prob, gpu, orc)
    return _cache[key]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def maxrel(a, b):
    """Largest entry-wise difference over the largest entry: a wrong value in
    one element is not diluted by the vector's length, as in rel()."""
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def oracle_rhs(prob, orc):
    """b of eqs. (appstokes1)-(appstokes2) times M from the oracle, element-major."""
    from oracle import ldg as oldg
    return orc.levels[0].P @ oldg.rhs(prob, orc.levels[0].ops)


@pytest.mark.parametrize("name", list(CASES))
def test_hierarchy_and_blocks(name):
    prob, gpu, orc = get(name)
    assert gpu.nlevels == len(orc.levels)
    assert gpu.n_snapped == orc.kernel_dim_bottom
    rng = np.random.default_rng(5)
    for l, lev in enumerate(orc.levels):
        nb, ne = lev.nb, lev.ne
        scale = abs(lev.A).max()
        els = range(ne) if ne <= 32 else rng.choice(ne, 24, replace=False)
        for i in els:
            row = lev.A[i * nb:(i + 1) * nb, :].toarray()
            cols = set(np.nonzero(np.abs(row).sum(0))[0] // nb) | {i}
            for j in cols:
                blk = gpu.ctx.get_block(l, int(i), int(j), nb)
                assert np.abs(blk - row[:, j * nb:(j + 1) * nb]).max() <= 1e-13 * scale


@pytest.mark.parametrize("name", list(CASES))
def test_colour_step_and_residual(name):
    prob, gpu, orc = get(name)
    rng = np.random.default_rng(11)
    n = prob.n_dofs
    x0 = rng.uniform(-1, 1, n)
    b = rng.uniform(-1, 1, n)
    sm = orc.sm[0]
    xd, bd = dev(x0), dev(b)
    xo = x0.copy()
    for c in range(sm.ncol):
        gpu.ctx.gs_colour(0, c, xd, bd)
        sm.colour_step(xo, b, c)
        xg = xd.cpu().numpy()
        assert rel(xg, xo) <= 1e-13 and maxrel(xg, xo) <= 1e-13
    r = torch.empty_like(xd)
    nrm = gpu.ctx.residual(xd, bd, r, want_norm=True)
    ro = orc.residual(0, xo, b)
    assert rel(r.cpu().numpy(), ro) <= 1e-12 and maxrel(r.cpu().numpy(), ro) <= 1e-12
    assert abs(nrm - np.linalg.norm(ro)) <= 1e-12 * np.linalg.norm(ro)


@pytest.mark.parametrize("name", ["periodic16p2", "stress16p3", "3d-mixed-p1"])
def test_transfers_and_bottom(name):
    prob, gpu, orc = get(name)
    rng = np.random.default_rng(3)
    for l in range(len(orc.levels) - 1):
        nf, nc = orc.levels[l].ne * orc.levels[l].nb, orc.levels[l + 1].ne * orc.levels[l + 1].nb
        r = rng.standard_normal(nf)
        rc = torch.zeros(nc, dtype=torch.float64, device="cuda")
        gpu.ctx.restrict(l, dev(r), rc)
        assert rel(rc.cpu().numpy(), orc.restrict(l, r)) <= 1e-14
        assert maxrel(rc.cpu().numpy(), orc.restrict(l, r)) <= 1e-14
        xc = rng.standard_normal(nc)
        x = rng.standard_normal(nf)
        xd = dev(x)
        gpu.ctx.prolong(l, dev(xc), xd)
        assert rel(xd.cpu().numpy(), x + orc.prolong(l, xc)) <= 1e-14
        assert maxrel(xd.cpu().numpy(), x + orc.prolong(l, xc)) <= 1e-14
    nbot = orc.levels[-1].ne * orc.levels[-1].nb
    bb = rng.standard_normal(nbot)
    xb = torch.zeros(nbot, dtype=torch.float64, device="cuda")
    gpu.ctx.bottom_solve(dev(bb), xb)
    assert rel(xb.cpu().numpy(), orc.bottom_solve(bb)) <= 1e-12
    assert maxrel(xb.cpu().numpy(), orc.bottom_solve(bb)) <= 1e-12


def trivial_kernel(prob, orc):
    """Orthonormal basis of the trivial null space among the constant fields
    (one per variable, mode 0 in every element; divided by the sqrt(mu)
    scaling when it is on): periodic constants of Section 3's footnote."""
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
    q, _ = np.linalg.qr(np.stack(cols, axis=1))
    return q


@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_iterates(name):
    """Algorithm 1 iterates x_k = V(x_{k-1}, b), k = 1..10, from x_0 = 0, for a
    consistent right-hand side (b orthogonal to the trivial kernel); iterates
    are compared modulo that kernel (they are unique only up to it)."""
    prob, gpu, orc = get(name)
    rng = np.random.default_rng(21)
    Z = trivial_kernel(prob, orc)
    b = rng.uniform(-1, 1, prob.n_dofs)
    b -= Z @ (Z.T @ b)
    bd = dev(b)
    xd = torch.zeros_like(bd)
    xo = np.zeros(prob.n_dofs)
    worst = worst_entry = 0.0
    for k in range(10):
        gpu.ctx.vcycle(xd, bd)
        orc.vcycle(xo, b)
        xg = xd.cpu().numpy()
        xg = xg - Z @ (Z.T @ xg)
        xr = xo - Z @ (Z.T @ xo)
        worst = max(worst, rel(xg, xr))
        worst_entry = max(worst_entry, maxrel(xg, xr))
    assert worst <= 1e-12, worst
    assert worst_entry <= 1e-12, worst_entry


@pytest.mark.parametrize("name", ["periodic16p2", "stress16p3", "dirichlet-rect", "3d-unsteady-p2"])
def test_solve_fp64_matches_oracle(name):
    prob, gpu, orc = get(name)
    b = gpu.rhs().ravel()
    bd = dev(b)
    xd = torch.zeros_like(bd)
    it, hist = gpu.ctx.solve(xd, bd, rtol=1e-10, maxit=100)
    xo, ho = orc.solve(b, rtol=1e-10, maxit=100)
    assert hist[-1] <= 1e-10
    assert abs(it - (len(ho) - 1)) <= 1
    assert rel(xd.cpu().numpy(), xo) <= 1e-11
    assert maxrel(xd.cpu().numpy(), xo) <= 1e-11


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_matches_oracle(name):
    """The library's right-hand side (stk_assemble_rhs, or stk_assemble_rhs2
    with interface jump data on the two-phase cases) equals the oracle's b of
    eqs. (appstokes1)-(appstokes2) times M entry by entry: volume forcing and
    divergence data, Dirichlet data with its penalty and lift terms
    (J_g, E_u,g(0)), stress data (J_h) and, across the interface, the jumps
    g and h with their viscosity-upwinded weights (eqs. govern2-govern3)."""
    prob, gpu, orc = get(name)
    b = gpu.rhs().ravel()
    bo = oracle_rhs(prob, orc)
    assert maxrel(b, bo) <= 1e-13, maxrel(b, bo)
    assert rel(b, bo) <= 1e-13


def test_large_bottom_takes_cusolver_and_matches_oracle():
    """The 2916-unknown bottom of the 6^3 p=2 problem is factorised by the
    equilibrated cuSOLVER path (not a host fallback), snaps exactly the
    kernel the oracle snaps, and solves like the oracle's pseudo-inverse."""
    prob, gpu, orc = get("3d-unsteady-6p2")
    assert gpu.ctx.info(native.INFO_BOTTOM_UNKNOWNS) == 27 * prob.nb == 2916
    assert gpu.ctx.info(native.INFO_BOTTOM_SOLVER) == native.BOTTOM_CUSOLVER
    assert gpu.n_snapped == orc.kernel_dim_bottom == 1
    rng = np.random.default_rng(9)
    for _ in range(2):
        bb = rng.standard_normal(2916)
        xb = torch.zeros(2916, dtype=torch.float64, device="cuda")
        gpu.ctx.bottom_solve(dev(bb), xb)
        xo = orc.bottom_solve(bb)
        assert rel(xb.cpu().numpy(), xo) <= 1e-12 and maxrel(xb.cpu().numpy(), xo) <= 1e-12


@pytest.mark.parametrize("precision", [native.FP32, native.BF16, native.FP16])
@pytest.mark.parametrize("name", ["stress16p3", "periodic16p2", "3d-unsteady-p2"])
def test_mixed_precision_refinement(name, precision):
    """Low-precision V-cycles inside FP64 refinement reach 1e-10 and the same
    solution as the FP64 path."""
    prob, gpu64, orc = get(name)
    _, gpu, _ = get(name, precision)
    b = gpu64.rhs().ravel()
    bd = dev(b)
    x64 = torch.zeros_like(bd)
    gpu64.ctx.solve(x64, bd, rtol=1e-10, maxit=100)
    x = torch.zeros_like(bd)
    it, hist = gpu.ctx.solve(x, bd, rtol=1e-10, maxit=200)
    assert hist[-1] <= 1e-10, hist
    assert rel(x.cpu().numpy(), x64.cpu().numpy()) <= 1e-8


STORAGE = {native.FP32: "fp32", native.BF16: "bf16", native.FP16: "fp16"}


@pytest.mark.parametrize("precision", [native.FP32, native.BF16, native.FP16])
@pytest.mark.parametrize("name", ["stress16p3", "3d-unsteady-p2"])
def test_low_precision_cycle_close_to_oracle_emulation(name, precision):
    """One low-precision cycle against the oracle with the same rounded
    blocks (FP32, BF16, or FP16 with per-sub-block / per-row power-of-two
    scales) and the in-cycle residual from them.  The library keeps FP32
    vectors and sums, the emulation FP64, so the bar is FP32-level agreement
    (amplified by the cycle)."""
    prob, gpu64, _ = get(name)
    _, gpu, _ = get(name, precision)
    orc = oracle_for(prob, storage=STORAGE[precision])
    b = gpu64.rhs().ravel()
    bd = dev(b)
    x = torch.zeros_like(bd)
    it, hist = gpu.ctx.solve(x, bd, rtol=1e-30, maxit=1)
    xo = orc.precondition(b)
    assert rel(x.cpu().numpy(), xo) <= 1e-4
    if precision != native.FP32:
        # and it is the rounded operator that is being emulated: the FP32 one differs more
        orc32 = oracle_for(prob, storage="fp32")
        assert rel(x.cpu().numpy(), orc32.precondition(b)) > 10 * rel(x.cpu().numpy(), xo)


@pytest.mark.parametrize("name", ["stress16p3", "periodic16p2", "dirichlet-rect", "3d-mixed-p1", "square-1e-3"])
def test_fp32_cycle_matches_float32_emulation(name):
    """One FP32 cycle (FP32-rounded blocks, FP32 vectors, FP32 sums) against
    the oracle's float32 emulation of the same cycle (precondition_fp32) and
    its FP64-vector emulation: within FP32 rounding noise of both, 3e-5
    relative and 5e-5 entry-wise.  (Measured: the GPU lies 4e-7 to 1.4e-5
    from the float32 emulation and 3e-7 to 9e-6 from the FP64-vector one; its
    fused multiply-adds round once per product and sum, numpy's float32 twice,
    so the FP64-vector emulation is the nearer of the two.)"""
    prob, gpu64, _ = get(name)
    _, gpu, _ = get(name, native.FP32)
    orc = oracle_for(prob, storage="fp32")
    b = gpu64.rhs().ravel()
    bd = dev(b)
    x = torch.zeros_like(bd)
    gpu.ctx.set_solver(native.RICHARDSON, 30)   # one outer step from zero is x = V(b)
    gpu.ctx.solve(x, bd, rtol=1e-30, maxit=1)
    xg = x.cpu().numpy()
    x32 = orc.precondition_fp32(b)
    x64 = orc.precondition(b)
    print(name, "fp32 emulation %.1e (entry-wise %.1e), fp64-vector emulation %.1e"
          % (rel(xg, x32), maxrel(xg, x32), rel(xg, x64)))
    assert rel(xg, x32) <= 3e-5 and maxrel(xg, x32) <= 5e-5
    assert rel(xg, x64) <= 3e-5 and maxrel(xg, x64) <= 5e-5


@pytest.mark.parametrize("name", ["stress16p3", "periodic16p2", "3d-mixed-p1"])
def test_fp16_colour_step_warp_and_wide_kernels(name):
    """FP16 colour steps of both kernels (one warp per element; one CTA per
    element) against the oracle's colour step with the same scaled FP16
    blocks, in FP32-level agreement."""
    prob, _, _ = get(name)
    _, gpu, _ = get(name, native.FP16)
    orc = oracle_for(prob, storage="fp16")
    sm = orc.sm[0]
    rng = np.random.default_rng(17)
    x0 = rng.uniform(-1, 1, prob.n_dofs).astype(np.float32).astype(np.float64)
    b = rng.uniform(-1, 1, prob.n_dofs).astype(np.float32).astype(np.float64)
    xo = x0.copy()
    for c in range(sm.ncol):
        sm.colour_step(xo, b, c)
    try:
        for wide in (0, 1 << 30):
            gpu.ctx.set_wide_launch(wide)
            xd = torch.from_numpy(x0).float().cuda()
            bd = torch.from_numpy(b).float().cuda()
            for c in range(sm.ncol):
                gpu.ctx.gs_colour_ex(0, c, native.FP16, xd, bd)
            assert rel(xd.double().cpu().numpy(), xo) <= 1e-4, wide
    finally:
        gpu.ctx.set_wide_launch(1024)


def _steps_and_residual(gpu, precision, x0, b):
    """Every colour step of level 0 from x0, then the residual of the result,
    as float32 arrays."""
    xd = torch.from_numpy(x0).float().cuda()
    bd = torch.from_numpy(b).float().cuda()
    for c in range(gpu.ctx.info(native.INFO_COLOURS)):
        gpu.ctx.gs_colour_ex(0, c, precision, xd, bd)
    r = torch.empty_like(xd)
    gpu.ctx.residual_ex(0, precision, xd, bd, r)
    torch.cuda.synchronize()
    return xd.cpu().numpy(), r.cpu().numpy()


def _with_variant(gpu, precision, variant, fn, shape=0):
    gpu.ctx.set_wide_launch(0)
    gpu.ctx.set_tuning(variant, precision, shape)
    try:
        return fn()
    finally:
        gpu.ctx.set_tuning(3, precision)   # the default for 16-bit records
        gpu.ctx.set_wide_launch(1024)


@pytest.mark.parametrize("warps", [1, 2, 4])
@pytest.mark.parametrize("precision", [native.FP16, native.BF16])
@pytest.mark.parametrize("name", ["stress16p3", "3d-mixed-p1"])
def test_staged_16bit_kernel_matches_oracle(name, precision, warps):
    """The warp kernel with the next element staged in shared memory (variant
    3, 16-bit records): its colour steps and residual agree with the plain
    warp kernel's to FP32 rounding (the same products; each coupling row
    summed as two halves of its columns), and its colour steps equal the
    oracle's colour step with the same rounded blocks to FP32 level."""
    prob, _, _ = get(name)
    _, gpu, _ = get(name, precision)
    orc = oracle_for(prob, storage="fp16" if precision == native.FP16 else "bf16")
    sm = orc.sm[0]
    rng = np.random.default_rng(23)
    x0 = rng.uniform(-1, 1, prob.n_dofs).astype(np.float32).astype(np.float64)
    b = rng.uniform(-1, 1, prob.n_dofs).astype(np.float32).astype(np.float64)
    xs, rs = _with_variant(gpu, precision, 3, lambda: _steps_and_residual(gpu, precision, x0, b), warps)
    xw, rw = _with_variant(gpu, precision, 2, lambda: _steps_and_residual(gpu, precision, x0, b))
    assert rel(xs, xw) <= 1e-5 and maxrel(xs, xw) <= 1e-5
    assert rel(rs, rw) <= 1e-5 and maxrel(rs, rw) <= 1e-5
    xo = x0.copy()
    for c in range(sm.ncol):
        sm.colour_step(xo, b, c)
    assert rel(xs, xo) <= 1e-4 and maxrel(xs, xo) <= 1e-3


@pytest.mark.parametrize("warps", [1, 2, 4])
@pytest.mark.parametrize("precision", [native.FP16, native.BF16])
def test_staged_16bit_kernel_on_many_elements_per_warp(precision, warps):
    """128 x 128, p = 3 viscous stress: each element slot of the staged kernel
    walks several elements per launch (4096 per colour over 152 x 10 slots),
    so every element's records are requested while the warp computes the
    one before.  Colour steps and residual agree with the plain warp kernel's
    to FP32 rounding."""
    prob = P.stress_variable_mu_2d(n=128, p=3)
    gpu = StokesMG(prob, precision=precision)
    try:
        rng = np.random.default_rng(29)
        x0 = rng.uniform(-1, 1, prob.n_dofs).astype(np.float32).astype(np.float64)
        b = rng.uniform(-1, 1, prob.n_dofs).astype(np.float32).astype(np.float64)
        xs, rs = _with_variant(gpu, precision, 3, lambda: _steps_and_residual(gpu, precision, x0, b), warps)
        xw, rw = _with_variant(gpu, precision, 2, lambda: _steps_and_residual(gpu, precision, x0, b))
        assert np.all(np.isfinite(xs)) and np.abs(xs - x0).max() > 0
        assert rel(xs, xw) <= 1e-5 and maxrel(xs, xw) <= 1e-5
        assert rel(rs, rw) <= 1e-5 and maxrel(rs, rw) <= 1e-5
    finally:
        gpu.close()


@pytest.mark.parametrize("wide", [0, 1024])
@pytest.mark.parametrize("precision", [native.FP16, native.BF16, native.FP32, native.FP64])
def test_launch_overlap_is_bit_identical(precision, wide):
    """Programmatic dependent launch of the element kernels
    (stk_set_launch_overlap): whole solves (V-cycles replayed from CUDA
    graphs, transfers, bottom solve; the staged kernel for 16-bit records,
    the warp kernel otherwise, and with wide = 1024 the one-CTA-per-element
    kernel on the coarse levels) give the same iterate bit for bit with the
    overlap on and off."""
    prob = P.stress_variable_mu_2d(n=64, p=3)
    gpu = StokesMG(prob, precision=precision)
    try:
        gpu.ctx.set_wide_launch(wide)
        gpu.ctx.set_solver(native.FGMRES, 30)
        b = torch.from_numpy(gpu.rhs().ravel()).cuda()
        out = []
        for on in (1, 0, 1):
            gpu.ctx.set_launch_overlap(on)
            x = torch.zeros_like(b)
            it, hist = gpu.ctx.solve(x, b, rtol=1e-10, maxit=100)
            out.append((it, x.cpu().numpy(), hist[-1]))
        assert out[0][0] == out[1][0] == out[2][0]
        assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][1], out[2][1])
        assert out[0][2] <= 1e-10
    finally:
        gpu.close()


def test_invalid_arguments_are_rejected():
    ctx = native.Context(0)
    with pytest.raises(native.StkError):
        ctx.set_mesh(2, (4, 4), (0, 0), (1, 1), (0, 1, 0, 0))      # periodic on one side only
    with pytest.raises(native.StkError):
        ctx.set_mesh(4, (4, 4, 4, 4), (0,) * 4, (1,) * 4, (0,) * 8)
    ctx.set_mesh(2, (4, 4), (0, 0), (1, 1), (0, 0, 0, 0))
    with pytest.raises(native.StkError):
        ctx.set_discretisation(0, 0)
    ctx.set_discretisation(2, 0)
    nv = ctx.num_points(native.PTS_VOLUME)
    ni = ctx.num_points(native.PTS_INTERIOR_FACE)
    with pytest.raises(native.StkError):
        ctx.set_viscosity(-np.ones(nv), np.ones(ni), np.zeros(0))  # mu must be positive
    with pytest.raises(native.StkError):
        x = torch.zeros(10, dtype=torch.float64, device="cuda")
        ctx.vcycle(x, x)                                             # not set up
    ctx.close()


@pytest.mark.parametrize("precision", [native.FP64, native.FP32, native.BF16, native.FP16])
@pytest.mark.parametrize("name", ["stress16p3", "periodic16p2", "3d-unsteady-p2"])
def test_fgmres_solve(name, precision):
    """Flexible GMRES with the V-cycle as right preconditioner (Section 3):
    reaches 1e-10 in FP64; in FP64 it follows the oracle's FGMRES."""
    prob, gpu64, orc = get(name)
    _, gpu, _ = get(name, precision)
    b = gpu64.rhs().ravel()
    bd = dev(b)
    x = torch.zeros_like(bd)
    gpu.ctx.set_solver(native.FGMRES, 30)
    try:
        it, hist = gpu.ctx.solve(x, bd, rtol=1e-10, maxit=200)
    finally:
        gpu.ctx.set_solver(native.RICHARDSON, 30)
    assert hist[-1] <= 1e-10, hist
    xo, ho = orc.fgmres(b, rtol=1e-10, maxit=200, restart=30)
    if precision == native.FP64:
        assert abs(it - (len(ho) - 1)) <= 1
        assert rel(x.cpu().numpy(), xo) <= 1e-9
    else:
        assert it <= (len(ho) - 1) + 3


@pytest.mark.parametrize("variant", [0, 1, 2, "wide"])
@pytest.mark.parametrize("name", ["stress16p3", "periodic16p2", "3d-mixed-p1"])
def test_kernel_variants_agree(name, variant):
    """All element-kernel variants (direct loads, bulk-copy ring, warp per
    element, and the one-CTA-per-element latency variant of small launches)
    give the oracle's colour step and residual in FP64."""
    prob, gpu, orc = get(name)
    if variant == "wide":
        gpu.ctx.set_tuning(2, native.FP64)
        gpu.ctx.set_wide_launch(1 << 30)
    else:
        gpu.ctx.set_tuning(variant, native.FP64)
        gpu.ctx.set_wide_launch(0)
    try:
        rng = np.random.default_rng(13)
        x0 = rng.uniform(-1, 1, prob.n_dofs)
        b = rng.uniform(-1, 1, prob.n_dofs)
        xd, bd = dev(x0), dev(b)
        xo = x0.copy()
        sm = orc.sm[0]
        for c in range(sm.ncol):
            gpu.ctx.gs_colour(0, c, xd, bd)
            sm.colour_step(xo, b, c)
        assert rel(xd.cpu().numpy(), xo) <= 1e-13
        r = torch.empty_like(xd)
        gpu.ctx.residual(xd, bd, r)
        assert rel(r.cpu().numpy(), orc.residual(0, xo, b)) <= 1e-12
    finally:
        gpu.ctx.set_tuning(2, native.FP64)
        gpu.ctx.set_wide_launch(1024)


@pytest.mark.parametrize("nrhs", [3, 8])
@pytest.mark.parametrize("name", ["stress16p3", "3d-mixed-p1", "3d-unsteady-p2"])
def test_multi_rhs_iteration_matches_oracle(name, nrhs):
    """One outer iteration for several right-hand sides at once equals, per
    right-hand side, x1 = x0 + V(0, b - A x0) of the oracle (FP64)."""
    prob, gpu, orc = get(name)
    rng = np.random.default_rng(31)
    X0 = rng.uniform(-1, 1, (nrhs, prob.n_dofs))
    B = rng.uniform(-1, 1, (nrhs, prob.n_dofs))
    Xd, Bd = dev(X0).reshape(nrhs, -1), dev(B).reshape(nrhs, -1)
    it, hist = gpu.ctx.solve_multi(Xd, Bd, nrhs, rtol=1e-30, maxit=1, inner=1)
    assert it == 1
    Xg = Xd.cpu().numpy()
    for q in range(nrhs):
        ref = X0[q] + orc.precondition(B[q] - orc.A @ X0[q])
        assert rel(Xg[q], ref) <= 1e-12


@pytest.mark.parametrize("precision,inner", [(native.FP64, 1), (native.FP32, 1), (native.FP32, 3), (native.BF16, 3)])
def test_multi_rhs_solve_converges(precision, inner):
    name = "stress16p3"
    prob, gpu64, _ = get(name)
    _, gpu, _ = get(name, precision)
    nrhs = 5
    rng = np.random.default_rng(8)
    B = rng.uniform(-1, 1, (nrhs, prob.n_dofs))
    Bd = dev(B).reshape(nrhs, -1)
    Xd = torch.zeros_like(Bd)
    it, hist = gpu.ctx.solve_multi(Xd, Bd, nrhs, rtol=1e-10, maxit=60, inner=inner)
    assert np.all(hist[-1] <= 1e-10), hist[-1]
    x1 = torch.zeros_like(Bd[1])
    gpu64.ctx.solve(x1, Bd[1].contiguous(), rtol=1e-12, maxit=200)
    assert rel(Xd[1].cpu().numpy(), x1.cpu().numpy()) <= 1e-8


@pytest.mark.parametrize("precision,method", [(native.FP64, native.FGMRES), (native.FP32, native.FGMRES),
                                              (native.FP32, native.FGMRES_IR)])
@pytest.mark.parametrize("name", ["stress16p3", "3d-unsteady-p2"])
def test_multi_rhs_fgmres_lockstep(name, precision, method):
    """Several right-hand sides by flexible GMRES in lockstep (one multi-RHS
    V-cycle per step; the refined variant with an FP32 Krylov matvec):
    every right-hand side reaches 1e-10, its solution is the
    single-right-hand-side solution (up to the kernel), and the step count is
    that of the slowest single solve (+-1; +-3 for the refined variant)."""
    prob, _, orc = get(name)
    _, gpu, _ = get(name, precision)
    nrhs = 6
    rng = np.random.default_rng(12)
    B = rng.uniform(-1, 1, (nrhs, prob.n_dofs))
    Z = trivial_kernel(prob, orc)   # consistent right-hand sides for singular (periodic) operators
    B -= (B @ Z) @ Z.T
    Bd = dev(B).reshape(nrhs, -1)
    Xd = torch.zeros_like(Bd)
    gpu.ctx.set_solver(method, 30)
    try:
        it, hist = gpu.ctx.solve_multi(Xd, Bd, nrhs, rtol=1e-10, maxit=80)
        assert np.all(hist[-1] <= 1e-10), hist[-1]
        singles = []
        for q in range(nrhs):
            x1 = torch.zeros_like(Bd[q])
            it1, h1 = gpu.ctx.solve(x1, Bd[q].contiguous(), rtol=1e-10, maxit=80)
            singles.append(it1)
            xa, xb = Xd[q].cpu().numpy(), x1.cpu().numpy()
            assert rel(xa - Z @ (Z.T @ xa), xb - Z @ (Z.T @ xb)) <= 1e-8   # unique up to the kernel
            r = torch.empty_like(x1)
            assert gpu.ctx.residual(Xd[q].contiguous(), Bd[q].contiguous(), r, want_norm=True) <= \
                1e-10 * np.linalg.norm(B[q])
        assert abs(it - max(singles)) <= (1 if method == native.FGMRES else 3), (it, singles)
    finally:
        gpu.ctx.set_solver(native.RICHARDSON, 30)


@pytest.mark.parametrize("name", ["stress16p3", "3d-mixed-p1", "3d-unsteady-p2"])
def test_multi_rhs_tensor_cores_match_cuda_cores(name):
    """Eight right-hand sides with FP32 blocks: the tensor-core kernels (3xTF32
    mma.sync; one warp per element, and four warps per element for small
    launches) and the CUDA-core kernel give the same outer iteration to
    FP32-level agreement, and all stay within 1e-4 of the oracle's cycle with
    FP32-rounded blocks."""
    prob, _, _ = get(name)
    _, gpu, _ = get(name, native.FP32)
    orc32 = oracle_for(prob, storage="fp32")
    nrhs = 8
    rng = np.random.default_rng(41)
    B = rng.uniform(-1, 1, (nrhs, prob.n_dofs))
    out = {}
    try:
        for key, on, small in (("warp", 1, 0), ("cta", 1, 1 << 30), ("cuda", 0, 1024)):
            gpu.ctx.set_mrhs_tensor(on)
            gpu.ctx.set_wide_launch(small)
            Xd = torch.zeros(nrhs, prob.n_dofs, dtype=torch.float64, device="cuda")
            gpu.ctx.solve_multi(Xd, dev(B).reshape(nrhs, -1), nrhs, rtol=1e-30, maxit=1, inner=1)
            out[key] = Xd.cpu().numpy()
    finally:
        gpu.ctx.set_mrhs_tensor(1)
        gpu.ctx.set_wide_launch(1024)
    for q in range(nrhs):
        ref = orc32.precondition(B[q])
        for key in ("warp", "cta"):
            assert rel(out[key][q], out["cuda"][q]) <= 1e-5, key
            assert rel(out[key][q], ref) <= 1e-4, key


def _learned_ctx():
    prob = P.stress_variable_mu_2d(n=16, p=3)
    gpu = StokesMG(prob, precision=native.FP32, nu=(3, 3))
    gpu.ctx.learn_setup(hidden=32, seed=5)
    return prob, gpu


def test_learned_features_and_mlp_match_oracle():
    from oracle import learned, ldg as oldg
    prob, gpu = _learned_ctx()
    nin, hid, nout, npar, _ = gpu.ctx.learn_sizes()
    w = gpu.ctx.learn_weights(npar).astype(np.float64)
    rng = np.random.default_rng(3)
    r = rng.standard_normal((prob.n_elements, prob.nb)).astype(np.float32)
    rd = torch.from_numpy(r.ravel()).cuda()
    y = torch.empty_like(rd)
    nrm = torch.empty(prob.n_elements, dtype=torch.float32, device="cuda")
    gpu.ctx.learn_infer(rd, y, nrm)
    mesh = oldg.Mesh(prob.d, prob.n, prob.lo, prob.hi, prob.bc)
    F, n_ref = learned.features(r.astype(np.float64), learned.face_neighbours(mesh))
    y_ref, _ = learned.forward(F, w, nin, hid, nout)
    assert rel(nrm.cpu().numpy(), n_ref) <= 1e-6
    assert rel(y.cpu().numpy().reshape(prob.n_elements, -1), y_ref) <= 1e-5
    gpu.close()


def test_learned_training_gradient_matches_oracle_backprop():
    """Loss ||r - A delta||^2/||r||^2 and its gradient on a stored residual
    state: GPU (FP32 blocks, FP32 kernels) against the oracle (FP64)."""
    from oracle import learned, ldg as oldg
    prob, gpu = _learned_ctx()
    gpu.ctx.learn_generate(nseeds=2, cycles=2, seed=11)
    nin, hid, nout, npar, states = gpu.ctx.learn_sizes()
    assert states == 4
    r = gpu.ctx.learn_state(1, prob.n_dofs).astype(np.float64).reshape(prob.n_elements, prob.nb)
    assert np.all(np.isfinite(r))
    loss, g = gpu.ctx.learn_grad(1, npar)
    w = gpu.ctx.learn_weights(npar).astype(np.float64)
    orc = multigrid.Multigrid(prob)
    mesh = oldg.Mesh(prob.d, prob.n, prob.lo, prob.hi, prob.bc)
    loss_ref, g_ref = learned.residual_loss_and_grad(orc.A, r, learned.face_neighbours(mesh), w, nin, hid, nout)
    assert abs(loss - loss_ref) <= 1e-4 * loss_ref
    assert rel(g, g_ref) <= 1e-3
    gpu.close()


def test_learned_smoother_solve_converges_and_is_judged():
    """Train on plain V-cycle pairs, enable, solve by iterative refinement:
    reaches 1e-10; after the two plain iterations that measure kappa every
    correction is kept or undone (or the correction is switched off after two
    undone in a row); a Krylov outer method is refused while it is enabled."""
    prob, gpu = _learned_ctx()
    gpu.ctx.learn_generate(nseeds=4, cycles=3, seed=1)
    loss0 = gpu.ctx.learn_train(epochs=1, batch=0, lr=1e-3, seed=2)
    loss1 = gpu.ctx.learn_train(epochs=20, batch=0, lr=1e-3, seed=3)
    assert np.isfinite(loss1) and loss1 <= loss0
    gpu.ctx.learn_enable(True)
    b = dev(gpu.rhs().ravel())
    x = torch.zeros_like(b)
    it, hist = gpu.ctx.solve(x, b, rtol=1e-10, maxit=100)
    assert hist[-1] <= 1e-10
    dec, ratio, kappa = gpu.ctx.learn_history()
    assert len(dec) == it and list(dec[:2]) == [-1, -1] and 0 < kappa < 1
    acc, rej = gpu.ctx.learn_stats()
    assert acc == int((dec == 1).sum()) and rej == int((dec == 0).sum())
    judged = [k for k in range(it) if dec[k] >= 0]
    assert all((ratio[k] < 1) == (dec[k] == 1) for k in judged)
    gpu.ctx.set_solver(native.FGMRES, 30)
    with pytest.raises(native.StkError):
        gpu.ctx.solve(x.zero_(), b, rtol=1e-10, maxit=100)
    gpu.close()


def test_learned_acceptance_matches_oracle():
    """The acceptance rule on the GPU (FP32 cycle and network) against the
    oracle's (FP32-rounded blocks, FP64 arithmetic, the same weights): the
    same kappa to 1e-5, the same decision in every judged iteration whose
    margin |ratio - 1| exceeds 1e-3 (up to the first closer call, after which
    the iterates may legitimately differ), and iteration counts within one."""
    from oracle import learned, ldg as oldg
    prob, gpu = _learned_ctx()
    gpu.ctx.learn_generate(nseeds=4, cycles=3, seed=1)
    gpu.ctx.learn_train(epochs=5, batch=0, lr=1e-3, seed=2)
    nin, hid, nout, npar, _ = gpu.ctx.learn_sizes()
    w = gpu.ctx.learn_weights(npar).astype(np.float64)
    gpu.ctx.learn_enable(True)
    b_host = gpu.rhs().ravel()
    b = dev(b_host)
    x = torch.zeros_like(b)
    it, hist = gpu.ctx.solve(x, b, rtol=1e-10, maxit=100)
    dec, ratio, kappa = gpu.ctx.learn_history()
    orc = multigrid.Multigrid(prob.with_(nu1=3, nu2=3), storage="fp32")   # the context's V(3,3)
    mesh = oldg.Mesh(prob.d, prob.n, prob.lo, prob.hi, prob.bc)
    xo, ho, dec_o, ratio_o, kappa_o = learned.solve_with_correction(orc, b_host, w, nin, hid, nout,
                                                                    learned.face_neighbours(mesh), rtol=1e-10,
                                                                    maxit=100)
    assert abs(kappa - kappa_o) <= 1e-5 * kappa_o
    compared = 0
    for k in range(min(len(dec), len(dec_o))):
        if dec_o[k] >= 0 and abs(ratio_o[k] - 1.0) <= 1e-3:
            break
        assert dec[k] == dec_o[k], (k, list(dec), dec_o)
        compared += 1
    assert compared >= 3
    assert abs(it - (len(ho) - 1)) <= 1 and hist[-1] <= 1e-10


def test_learned_supervised_gradient_matches_oracle():
    """The supervised objective (MSE of delta_i / ||r_i|| against the
    normalised error e_i / ||r_i|| of the stored plain-cycle states): loss and
    back-propagated gradient on a stored state equal the oracle's
    loss_and_grad on the same residual, error and weights."""
    from oracle import learned, ldg as oldg
    prob, gpu = _learned_ctx()
    gpu.ctx.learn_generate(nseeds=2, cycles=2, seed=11)
    gpu.ctx.learn_objective(1)
    nin, hid, nout, npar, states = gpu.ctx.learn_sizes()
    r = gpu.ctx.learn_state(2, prob.n_dofs).astype(np.float64).reshape(prob.n_elements, prob.nb)
    e = gpu.ctx.learn_error_state(2, prob.n_dofs).astype(np.float64).reshape(prob.n_elements, prob.nb)
    assert np.all(np.isfinite(e)) and np.abs(e).max() > 0
    loss, g = gpu.ctx.learn_grad(2, npar)
    w = gpu.ctx.learn_weights(npar).astype(np.float64)
    mesh = oldg.Mesh(prob.d, prob.n, prob.lo, prob.hi, prob.bc)
    F, nrm = learned.features(r, learned.face_neighbours(mesh))
    T = e / (nrm[:, None] + 1e-30)
    loss_ref, g_ref = learned.loss_and_grad(F, T, w, nin, hid, nout)
    assert abs(loss - loss_ref) <= 1e-4 * loss_ref
    assert rel(g, g_ref) <= 1e-3
    loss_tr = gpu.ctx.learn_train(epochs=3, batch=0, lr=1e-3, seed=5)
    assert np.isfinite(loss_tr)
    gpu.close()


@pytest.mark.parametrize("precision", [native.FP32, native.BF16, native.FP16])
@pytest.mark.parametrize("name", ["stress16p3", "3d-unsteady-p2"])
def test_fgmres_refined_variant(name, precision):
    """Krylov matvec on FP32 blocks (FP32 or BF16 cycle) with FP64 restarts
    still reaches 1e-10 on the FP64 residual and the FP64 solution."""
    prob, gpu64, _ = get(name)
    _, gpu, _ = get(name, precision)
    b = dev(gpu64.rhs().ravel())
    x64 = torch.zeros_like(b)
    gpu64.ctx.solve(x64, b, rtol=1e-11, maxit=200)
    x = torch.zeros_like(b)
    gpu.ctx.set_solver(native.FGMRES_IR, 30)
    try:
        it, hist = gpu.ctx.solve(x, b, rtol=1e-10, maxit=200)
    finally:
        gpu.ctx.set_solver(native.RICHARDSON, 30)
    assert hist[-1] <= 1e-10, hist
    assert rel(x.cpu().numpy(), x64.cpu().numpy()) <= 1e-8



@pytest.mark.parametrize("name", ["square-1e-3", "square-1e3-p3"])
def test_multiphase_colours_and_solve(name):
    """Grid-aligned two-phase problem (Section 5.6): the library's greedy
    colouring equals the oracle's; the scaled system solved by FGMRES gives the
    oracle's solution, and the unscaled velocity matches the manufactured one."""
    prob, gpu, orc = get(name)
    for l in range(len(orc.levels) - 1):
        assert np.array_equal(gpu.ctx.get_colours(l, orc.levels[l].ne), orc.levels[l].mesh.colour())
    D = gpu.scaling().ravel()
    np.testing.assert_allclose(D, orc.levels[0].D, rtol=1e-14)
    b = D * gpu.rhs().ravel()
    bd = dev(b)
    x = torch.zeros_like(bd)
    gpu.ctx.set_solver(native.FGMRES, 40)
    try:
        it, hist = gpu.ctx.solve(x, bd, rtol=1e-11, maxit=100)
    finally:
        gpu.ctx.set_solver(native.RICHARDSON, 30)
    assert hist[-1] <= 1e-11
    xo, ho = orc.fgmres(b, rtol=1e-11, maxit=100, restart=40)
    assert abs(it - (len(ho) - 1)) <= 1
    assert rel(x.cpu().numpy(), xo) <= 1e-9
    # unscaled velocity x = D x~ against the manufactured solution: the same
    # discretisation error as the oracle's solution (whose order p+1 the
    # oracle pins fix), below 1e-3 relative on both meshes
    eg = velocity_error(prob, orc, D * x.cpu().numpy())
    eo = velocity_error(prob, orc, orc.unscale(xo))
    assert np.all(eg <= 1e-3), eg
    np.testing.assert_allclose(eg, eo, rtol=1e-6)


def velocity_error(prob, orc, x):
    """Relative L2 error of each velocity component of the element-major
    coefficients x against prob.exact.u, after removing the constant (the
    periodic kernel); Gauss rule of p+3 points per axis."""
    from oracle import basis as obasis
    lev = orc.levels[0]
    mesh, d, p, s = lev.mesh, prob.d, prob.p, lev.s
    q = p + 3
    xv, wv = mesh.volume_points(q)
    Phi = obasis.tensor_basis(d, p, q)
    vals = np.einsum("qa,eva->eqv", Phi, x.reshape(mesh.ne, d + 1, s))
    ue = prob.exact.u(xv)
    out = []
    for v in range(d):
        err = vals[..., v] - ue[..., v]
        err = err - (err * wv).sum() / (wv.sum() * mesh.ne)
        out.append(np.sqrt((err ** 2 * wv).sum() / (ue[..., v] ** 2 * wv).sum()))
    return np.array(out)


@pytest.mark.parametrize("precision", [native.FP64, native.FP32])
def test_autotune_keeps_results(precision):
    """The autotuner (launch shapes timed on the context's own records) picks
    valid shapes, and afterwards the FP64 V-cycle iterates still match the
    oracle's to 1e-12 and a low-precision solve still reaches 1e-10."""
    name = "stress16p3"
    prob, _, orc = get(name)
    gpu = StokesMG(prob, precision=precision)
    try:
        choice, best = gpu.ctx.autotune()
        assert choice["variant"] in (0, 2) and choice["variant_fp64"] in (0, 2)
        assert choice["ctas_cycle"] in (2, 3, 4, 6, 8) and choice["ctas_fp64"] in (2, 3, 4, 6, 8)
        assert choice["wide_max"] >= 0 and best[0] > 0 and best[1] > 0
        rng = np.random.default_rng(23)
        b = rng.uniform(-1, 1, prob.n_dofs)
        if precision == native.FP64:
            xd, bd = torch.zeros(prob.n_dofs, dtype=torch.float64, device="cuda"), dev(b)
            xo = np.zeros(prob.n_dofs)
            for _ in range(5):
                gpu.ctx.vcycle(xd, bd)
                orc.vcycle(xo, b)
            assert rel(xd.cpu().numpy(), xo) <= 1e-12
        else:
            bd = dev(gpu.rhs().ravel())
            x = torch.zeros_like(bd)
            it, hist = gpu.ctx.solve(x, bd, rtol=1e-10, maxit=100)
            assert hist[-1] <= 1e-10
    finally:
        gpu.close()


BATCH = [(8, 2, 0, native.FP32), (16, 3, 1, native.FP64), (12, 2, 2, native.FP32), (16, 2, 3, native.FP16),
         (8, 3, 4, native.FP32), (24, 2, 5, native.BF16)]


def test_solve_batch_matches_individual_solves():
    """A batch of independent unsteady viscous-stress problems of different
    sizes, degrees and storage precisions solved concurrently
    (stk_solve_batch, four host threads) gives every problem what solving it
    alone gives: the same iteration count and solution, at 1e-10."""
    gpus = []
    try:
        for n, p, seed, prec in BATCH:
            g = StokesMG(P.unsteady_stress_2d(n=n, p=p, seed=seed), precision=prec)
            g.ctx.set_solver(native.FGMRES, 30)
            gpus.append(g)
        bs = [dev(g.rhs().ravel()) for g in gpus]
        xs = [torch.zeros_like(b) for b in bs]
        its, status = native.solve_batch([g.ctx for g in gpus], xs, bs, rtol=1e-10, maxit=100, threads=4)
        assert status == [native.STK_OK] * len(gpus)
        for g, b, x, it in zip(gpus, bs, xs, its):
            x1 = torch.zeros_like(b)
            it1, hist = g.ctx.solve(x1, b, rtol=1e-10, maxit=100)
            assert hist[-1] <= 1e-10 and abs(it1 - it) <= 1, (it1, it)
            assert rel(x.cpu().numpy(), x1.cpu().numpy()) <= 1e-9
            r = torch.empty_like(b)
            assert g.ctx.residual(x, b, r, want_norm=True) <= 1e-10 * torch.linalg.norm(b).item()
        with pytest.raises(native.StkError):   # one context twice in a batch is refused by the library
            native.solve_batch([gpus[0].ctx, gpus[0].ctx], [xs[0], xs[0]], [bs[0], bs[0]])
        with pytest.raises(ValueError):        # vectors of another problem's size, by the binding
            native.solve_batch([gpus[0].ctx, gpus[0].ctx], xs[:2], bs[:2])
    finally:
        for g in gpus:
            g.close()


def test_solve_batch_several_right_hand_sides():
    """The batch with three right-hand sides per problem runs stk_solve_multi
    for each problem; every right-hand side reaches 1e-10."""
    gpus = []
    try:
        for n, p, seed, prec in BATCH[:3]:
            if prec == native.FP16:
                continue
            gpus.append(StokesMG(P.unsteady_stress_2d(n=n, p=p, seed=seed), precision=prec))
        rng = np.random.default_rng(31)
        bs = [dev(rng.uniform(-1, 1, 3 * g.prob.n_dofs)) for g in gpus]
        xs = [torch.zeros_like(b) for b in bs]
        its, status = native.solve_batch([g.ctx for g in gpus], xs, bs, nrhs=3, rtol=1e-10, maxit=100, inner=3)
        for g, b, x in zip(gpus, bs, xs):
            nd = g.prob.n_dofs
            for q in range(3):
                r = torch.empty(nd, dtype=torch.float64, device="cuda")
                nrm = g.ctx.residual(x[q * nd:(q + 1) * nd], b[q * nd:(q + 1) * nd], r, want_norm=True)
                assert nrm <= 1e-10 * torch.linalg.norm(b[q * nd:(q + 1) * nd]).item()
    finally:
        for g in gpus:
            g.close()


@pytest.mark.parametrize("precision", [native.FP32, native.BF16, native.FP16])
@pytest.mark.parametrize("name", ["stress16p3", "3d-unsteady-p2", "square-1e3-p3"])
def test_fgmres_double_float_matvec(name, precision):
    """Flexible GMRES with its matvec on the FP32 units (FP32 records plus
    their FP32 remainders, exact products, two-sum accumulation) follows the
    FP64-matvec FGMRES: the same iteration count (+-1 under 16-bit cycles),
    1e-10 reached, for FP32 cycles the same residual history to 1e-5
    relative in every entry above 1e-9 (the cycle turns the matvecs' ~1e-14
    differences into ~1e-8 ones in its output, more under a 1e3 viscosity
    contrast) and the same solution to 1e-8."""
    prob, gpu64, _ = get(name)
    _, gpu, _ = get(name, precision)
    b = gpu64.rhs().ravel()
    if prob.scale_mu:
        b = gpu64.scaling().ravel() * b
    bd = dev(b)
    gpu.ctx.set_solver(native.FGMRES, 30)
    runs = {}
    try:
        for on in (0, 1):
            gpu.ctx.set_df_matvec(on)
            x = torch.zeros_like(bd)
            it, hist = gpu.ctx.solve(x, bd, rtol=1e-10, maxit=100)
            runs[on] = (it, np.asarray(hist), x.cpu().numpy())
    finally:
        gpu.ctx.set_df_matvec(1)
        gpu.ctx.set_solver(native.RICHARDSON, 30)
    (it0, h0, x0), (it1, h1, x1) = runs[0], runs[1]
    assert abs(it0 - it1) <= (0 if precision == native.FP32 else 1) and h1[-1] <= 1e-10, (it0, it1, h1[-1])
    if precision == native.FP32:   # 16-bit cycles amplify the perturbation further
        big = h0 > 1e-9
        assert np.all(np.abs(h1[big] - h0[big]) <= 1e-5 * h0[big] + 1e-13)
    Z = trivial_kernel(prob, get(name)[2])
    assert rel(x1 - Z @ (Z.T @ x1), x0 - Z @ (Z.T @ x0)) <= 1e-8


@pytest.mark.parametrize("shape", [(2, 1, 64), (1, 2, 64), (3, 2, 6)])
@pytest.mark.parametrize("name", ["stress16p3", "periodic16p2", "3d-unsteady-p2"])
def test_cycle_shapes_match_oracle(name, shape):
    """W-cycles and variable V-cycles (Section 6) in FP64: four cycle iterates
    (modulo the trivial kernel), one outer iteration for three right-hand sides
    at once, and the graph-replayed solve equal the oracle's with the same
    cycle shape; the shape is set after earlier solves, so cached graphs must
    be rebuilt."""
    prob, gpu, orc = get(name)
    rng = np.random.default_rng(41)
    Z = trivial_kernel(prob, orc)
    b = rng.uniform(-1, 1, prob.n_dofs)
    b -= Z @ (Z.T @ b)
    gpu.ctx.set_cycle_shape(*shape)
    orc.gamma, orc.growth, orc.max_sweeps = shape
    try:
        bd = dev(b)
        xd = torch.zeros_like(bd)
        xo = np.zeros(prob.n_dofs)
        for k in range(4):
            gpu.ctx.vcycle(xd, bd)
            orc.vcycle(xo, b)
            xg = xd.cpu().numpy()
            assert rel(xg - Z @ (Z.T @ xg), xo - Z @ (Z.T @ xo)) <= 1e-12, k
        X0 = rng.uniform(-1, 1, (3, prob.n_dofs))
        B = rng.uniform(-1, 1, (3, prob.n_dofs))
        Xd, Bd = dev(X0).reshape(3, -1), dev(B).reshape(3, -1)
        it, _ = gpu.ctx.solve_multi(Xd, Bd, 3, rtol=1e-30, maxit=1, inner=1)
        assert it == 1
        Xg = Xd.cpu().numpy()
        for q in range(3):
            assert rel(Xg[q], X0[q] + orc.precondition(B[q] - orc.A @ X0[q])) <= 1e-12, q
        bs = gpu.rhs().ravel()
        xd = torch.zeros_like(dev(bs))
        it, hist = gpu.ctx.solve(xd, dev(bs), rtol=1e-10, maxit=100)
        xo, ho = orc.solve(bs, rtol=1e-10, maxit=100)
        assert hist[-1] <= 1e-10 and abs(it - (len(ho) - 1)) <= 1
        assert rel(xd.cpu().numpy(), xo) <= 1e-11
    finally:
        gpu.ctx.set_cycle_shape(1, 1, 64)
        orc.gamma, orc.growth, orc.max_sweeps = 1, 1, 64


@pytest.mark.parametrize("precision", [native.FP32, native.FP16])
def test_w_cycle_low_precision_solve(precision):
    """A W-cycle of FP32 / scaled-FP16 blocks inside FGMRES reaches 1e-10 in no
    more iterations than the V-cycle of the same blocks, and a bad shape is
    rejected."""
    prob, gpu, _ = get("stress16p3", precision)
    b = dev(gpu.rhs().ravel())
    its = {}
    gpu.ctx.set_solver(native.FGMRES, 30)
    try:
        for shape in [(1, 1, 64), (2, 1, 64)]:
            gpu.ctx.set_cycle_shape(*shape)
            x = torch.zeros_like(b)
            its[shape], hist = gpu.ctx.solve(x, b, rtol=1e-10, maxit=60)
            assert hist[-1] <= 1e-10, shape
    finally:
        gpu.ctx.set_cycle_shape(1, 1, 64)
        gpu.ctx.set_solver(native.RICHARDSON, 30)
    assert its[(2, 1, 64)] <= its[(1, 1, 64)], its
    for bad in [(0, 1, 64), (4, 1, 64), (1, 0, 64), (1, 5, 64), (1, 1, 0), (1, 1, 257)]:
        with pytest.raises(RuntimeError):
            gpu.ctx.set_cycle_shape(*bad)


@pytest.mark.parametrize("name", ["periodic16p2", "stress16p3", "3d-unsteady-p2"])
def test_gmres_rho_matches_oracle(name):
    """eq. (rho) on the GPU (stk_gmres_rho: left-preconditioned GMRES on
    V A x = 0 from a random field, FP64 cycles) equals the oracle's: the same
    iteration count, rho, residual history and Arnoldi matrix."""
    prob, gpu, orc = get(name)
    x0 = P.random_vector(prob.n_elements, prob.nb, seed=1).ravel()
    rho, n, hist, H = gpu.ctx.gmres_rho(dev(x0), 1e-8, 100)
    rho_o, n_o, hist_o, H_o = orc.gmres_rho(x0, maxit=100, details=True)
    assert n == n_o and n < 100
    assert abs(rho - rho_o) <= 1e-9 * rho_o
    np.testing.assert_allclose(hist, hist_o, rtol=1e-8, atol=1e-15)
    # The Arnoldi basis is sensitive to rounding: each step multiplies the
    # previous steps' differences (here the library's classical Gram-Schmidt
    # done twice against the oracle's modified Gram-Schmidt, and 1e-13 cycle
    # differences) by up to the ratio of H's largest entries to its
    # subdiagonal (~10-50 on these operators); after n <= 12 steps the
    # entries agree to ~1e-8, so H is held to 1e-6 and its own least-squares
    # residuals to the history it produced.
    assert rel(H[: n + 1, :n], H_o[: n + 1, :n]) <= 1e-6
    e1 = np.zeros(n + 1)
    e1[0] = 1.0
    for k in range(1, n + 1):
        y = np.linalg.lstsq(H[: k + 1, :k], e1[: k + 1], rcond=None)[0]
        assert abs(np.linalg.norm(e1[: k + 1] - H[: k + 1, :k] @ y) - hist[k]) <= 1e-9 * hist[k]


def test_tau_sweep_valley_contains_table1_tau():
    """Section 4's tau sweep through the C ABI on the periodic 2D standard
    form, p = 2, 32 x 32, V(3,3): rho(tau) has an interior minimum (the
    valley), Table 1's tau lies within the 12.5 % window of that minimum
    (rho <= (min rho)^(8/9)), and rho at Table 1's tau equals the oracle's."""
    from paper_1911_05888_gb300 import tau as T
    taus, rhos, its = T.sweep(0, 2, 2, 32, per_octave=4, octaves=1)
    k = int(np.argmin(rhos))
    assert 0 < k < len(rhos) - 1, list(zip(taus, rhos))
    mid = len(rhos) // 2
    assert rhos[mid] <= rhos.min() ** (1 - T.EPS)
    q = P.generic(2, 32, 2, 0, [P.PERIODIC] * 4, nu=(3, 3), tau=taus[mid])
    x0 = P.random_vector(q.n_elements, q.nb, seed=1).ravel()
    rho_o, n_o = oracle_for(q).gmres_rho(x0, maxit=100)
    assert its[mid] == n_o and abs(rhos[mid] - rho_o) <= 1e-9 * rho_o


@pytest.mark.parametrize("name", ["periodic16p2", "dirichlet-rect", "3d-unsteady-p2"])
def test_colouring_modes(name):
    """Standard form (Section 3's block GS with a valid multi-colouring): by
    default the library colours every smoothing level with the checkerboard
    (two colours; the oracle's colour_two), and on request with the 2^d parity
    colours; in both modes the level colours equal the oracle's and four
    V-cycle iterates match the oracle with the same colouring to 1e-12."""
    prob, gpu, orc = get(name)
    assert gpu.ctx.info(native.INFO_COLOURS) == 2
    for l in range(len(orc.levels) - 1):
        assert np.array_equal(gpu.ctx.get_colours(l, orc.levels[l].ne), orc.levels[l].mesh.colour_two())
    par = StokesMG(prob, colouring=native.COLOURS_PARITY)
    try:
        orc_par = multigrid.Multigrid(prob, levels=orc.levels, injections=orc.I)
        assert par.ctx.info(native.INFO_COLOURS) == 2 ** prob.d
        for l in range(len(orc.levels) - 1):
            assert np.array_equal(par.ctx.get_colours(l, orc.levels[l].ne), orc.levels[l].mesh.colour())
        rng = np.random.default_rng(2)
        Z = trivial_kernel(prob, orc)
        b = rng.uniform(-1, 1, prob.n_dofs)
        b -= Z @ (Z.T @ b)
        for g, o in ((gpu, orc), (par, orc_par)):
            xd, xo = torch.zeros(prob.n_dofs, dtype=torch.float64, device="cuda"), np.zeros(prob.n_dofs)
            for _ in range(4):
                g.ctx.vcycle(xd, dev(b))
                o.vcycle(xo, b)
                xg = xd.cpu().numpy()
                xg, xr = xg - Z @ (Z.T @ xg), xo - Z @ (Z.T @ xo)
                assert rel(xg, xr) <= 1e-12 and maxrel(xg, xr) <= 1e-12
    finally:
        par.close()


def test_checkerboard_refused_for_viscous_stress_form():
    """The viscous-stress form couples diagonal neighbours, which the
    checkerboard puts in one colour: setup refuses it."""
    with pytest.raises(native.StkError):
        StokesMG(CASES["stress16p3"](), colouring=native.COLOURS_CHECKERBOARD)


EXTREME = {
    "square-1e-6": lambda: P.square_interface(n=16, p=2, mu_inner=1e-6),
    "square-1e6-p3": lambda: P.square_interface(n=8, p=3, mu_inner=1e6),
}


@pytest.mark.parametrize("name", list(EXTREME))
def test_multiphase_extreme_viscosity_ratios(name):
    """Section 5.6's square interface at viscosity ratios 1e-6 and 1e6: the
    library's greedy colours, sqrt(mu) scaling and right-hand side with jump
    data equal the oracle's (1e-13 / 1e-14 / 1e-13), ten V-cycle iterates
    agree to max(1e-12, 1e-16 cond(A_bottom)), and FGMRES reaches 1e-11 on the
    scaled system with the oracle's iteration count and a velocity of the same
    discretisation error below 1e-3.  The iterate tolerance: the sqrt(mu)
    scaling leaves the element blocks as well conditioned as at ratio 1
    (cond(A_ii) <= 1.5e6 on both), but the bottom operator of the 1e6 case has
    cond 1.8e8, and the bottom solve multiplies the rounding-level difference
    of its right-hand side (the two sides sum in different orders) by it."""
    prob = EXTREME[name]()
    gpu = StokesMG(prob)
    orc = oracle_for(prob)
    try:
        for l in range(len(orc.levels) - 1):
            assert np.array_equal(gpu.ctx.get_colours(l, orc.levels[l].ne), orc.levels[l].mesh.colour())
        D = gpu.scaling().ravel()
        np.testing.assert_allclose(D, orc.levels[0].D, rtol=1e-14)
        b = gpu.rhs().ravel()
        bo = oracle_rhs(prob, orc)
        assert maxrel(b, bo) <= 1e-13
        Z = trivial_kernel(prob, orc)
        rng = np.random.default_rng(21)
        bs = rng.uniform(-1, 1, prob.n_dofs)
        bs -= Z @ (Z.T @ bs)
        lam = np.abs(np.linalg.eigvalsh(orc.levels[-1].A.toarray()))
        lam = lam[lam > 1e-10 * lam.max()]
        tol = max(1e-12, 1e-16 * lam.max() / lam.min())
        xd = torch.zeros(prob.n_dofs, dtype=torch.float64, device="cuda")
        xo = np.zeros(prob.n_dofs)
        for k in range(10):
            gpu.ctx.vcycle(xd, dev(bs))
            orc.vcycle(xo, bs)
            xg = xd.cpu().numpy()
            assert rel(xg - Z @ (Z.T @ xg), xo - Z @ (Z.T @ xo)) <= tol, (k, tol)
        bsc = D * b
        x = torch.zeros(prob.n_dofs, dtype=torch.float64, device="cuda")
        gpu.ctx.set_solver(native.FGMRES, 40)
        it, hist = gpu.ctx.solve(x, dev(bsc), rtol=1e-11, maxit=100)
        assert hist[-1] <= 1e-11
        xo, ho = orc.fgmres(bsc, rtol=1e-11, maxit=100, restart=40)
        assert abs(it - (len(ho) - 1)) <= 1
        eg = velocity_error(prob, orc, D * x.cpu().numpy())
        eo = velocity_error(prob, orc, orc.unscale(xo))
        assert np.all(eg <= 1e-3), eg
        np.testing.assert_allclose(eg, eo, rtol=1e-6)
    finally:
        gpu.close()


@pytest.mark.parametrize("name,bottom,levels", [("stress16p3", 3072, 2), ("periodic16p2", 1728, 2),
                                                ("dirichlet-rect", 648, 2)])
def test_earlier_bottom_matches_oracle(name, bottom, levels):
    """A hierarchy stopped early (stk_set_bottom): the bottom level is the
    first coarse level with at most `bottom` unknowns, solved by the dense
    pseudo-inverse (cuSOLVER above 1200 unknowns), and ten V-cycle iterates
    equal the oracle's with the same number of levels to 1e-12."""
    prob = CASES[name]()
    gpu = StokesMG(prob, bottom_max=bottom)
    orc = oracle_for(prob, max_levels=levels)
    try:
        assert gpu.nlevels == len(orc.levels) == levels
        nbot = orc.levels[-1].ne * orc.levels[-1].nb
        assert gpu.ctx.info(native.INFO_BOTTOM_UNKNOWNS) == nbot <= bottom
        assert gpu.ctx.info(native.INFO_BOTTOM_SOLVER) == (native.BOTTOM_CUSOLVER if nbot > 1200 else
                                                           native.BOTTOM_HOST_QR if nbot > 300 else native.BOTTOM_JACOBI)
        assert gpu.n_snapped == orc.kernel_dim_bottom
        Z = trivial_kernel(prob, orc)
        b = np.random.default_rng(21).uniform(-1, 1, prob.n_dofs)
        b -= Z @ (Z.T @ b)
        xd = torch.zeros(prob.n_dofs, dtype=torch.float64, device="cuda")
        xo = np.zeros(prob.n_dofs)
        for k in range(10):
            gpu.ctx.vcycle(xd, dev(b))
            orc.vcycle(xo, b)
            xg = xd.cpu().numpy()
            assert rel(xg - Z @ (Z.T @ xg), xo - Z @ (Z.T @ xo)) <= 1e-12, k
    finally:
        gpu.close()
