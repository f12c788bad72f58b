"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, invariants (symmetry, kernel dimension), convergence orders quoted in
the text, the equivalence of operator coarsening with direct assembly, a dense
direct solve, and the tau / rho statements of Tables 1-2 and Sections 4-5.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1911_05888_gb300 import problems as P
from oracle import basis, hierarchy, ldg, multigrid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ----------------------------------------------------------------- basis ----

@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_legendre_orthonormal(p):
    np.testing.assert_allclose(basis.mass_1d(p), 2 * np.eye(p + 1), atol=1e-13)


def test_closed_forms_p1():
    # psi_0 = 1, psi_1 = sqrt(3) xi:  int psi_0 psi_1' = 2 sqrt(3), int psi_1 psi_1' = 0.
    K = basis.deriv_1d(1)
    np.testing.assert_allclose(K, [[0, 2 * np.sqrt(3)], [0, 0]], atol=1e-14)
    # psi_1((xi - 1)/2) = psi_1(xi)/2 - sqrt(3)/2 psi_0 on the lower child.
    P0 = basis.child_1d(1, 0)
    np.testing.assert_allclose(P0, [[1, -np.sqrt(3) / 2], [0, 0.5]], atol=1e-14)
    np.testing.assert_allclose(basis.trace_1d(1, -1), [1, -np.sqrt(3)], atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_injection_reproduces_coarse_polynomial(p):
    rng = np.random.default_rng(0)
    c = rng.standard_normal(p + 1)
    xi = np.linspace(-1, 1, 7)
    for child in (0, 1):
        fine = basis.child_1d(p, child) @ c
        coarse_at = basis.psi(p, (xi + 2 * child - 1) / 2) @ c
        np.testing.assert_allclose(basis.psi(p, xi) @ fine, coarse_at, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_derivative_matrix_integrates_by_parts(p):
    K = basis.deriv_1d(p)
    tp, tm = basis.trace_1d(p, 1), basis.trace_1d(p, -1)
    np.testing.assert_allclose(K + K.T, np.outer(tp, tp) - np.outer(tm, tm), atol=1e-12)


# --------------------------------------------------------- operator pins ----

def _problems_small():
    return [
        P.periodic_standard_2d(n=4, p=2),
        P.generic(2, 4, 2, 0, [P.DIRICHLET] * 4),
        P.generic(2, 4, 1, 1, [P.STRESS] * 4),
        P.stress_variable_mu_2d(n=4, p=2),
        P.generic(3, 4, 1, 0, [P.PERIODIC] * 6),
        P.generic(3, 4, 1, 1, [P.DIRICHLET, P.STRESS] * 3),
        P.unsteady_periodic_3d(n=4, p=1, re=10.0),
    ]


@pytest.mark.parametrize("prob", _problems_small(), ids=lambda q: q.name or str(q.bc))
def test_symmetry(prob):
    levels, _ = hierarchy.build_hierarchy(prob)
    for lev in levels:
        A = lev.A
        assert abs(A - A.T).max() <= 1e-13 * abs(A).max()


@pytest.mark.parametrize("prob,dim", [
    (P.periodic_standard_2d(n=4, p=2), 3),                          # constant u, constant p
    (P.generic(2, 4, 2, 0, [P.DIRICHLET] * 4), 1),                  # constant p
    (P.generic(2, 4, 2, 1, [P.STRESS] * 4), 3),                     # 2 translations + rotation
    (P.generic(2, 4, 1, 0, [P.DIRICHLET] * 3 + [P.STRESS]), 0),
    (P.generic(3, 2, 1, 0, [P.PERIODIC] * 6), 4),
    (P.unsteady_periodic_3d(n=2, p=1, re=10.0), 1),                 # mass term removes constant u
])
def test_kernel_dimension(prob, dim):
    lev = hierarchy.build_hierarchy(prob, max_levels=1)[0][0]
    lam = np.linalg.eigvalsh(lev.A.toarray())
    assert int((np.abs(lam) <= 1e-10 * np.abs(lam).max()).sum()) == dim


def test_rotation_in_stress_kernel():
    """gamma = 1 with stress conditions: u = (-y, x), p = 0 is a null vector
    (Section 3 footnote on the trivial kernel)."""
    prob = P.generic(2, 4, 1, 1, [P.STRESS] * 4)
    lev = hierarchy.build_hierarchy(prob, max_levels=1)[0][0]
    mesh, s, nb = lev.mesh, lev.s, lev.nb
    x = np.zeros((mesh.ne, nb))
    # L2 projection of (-y, x) on Q_1: mode 0 = value at centre, x-linear mode
    # psi_1(xi_x) = sqrt(3) xi_x with x = c + h xi / 2.
    for e in range(mesh.ne):
        cx, cy = mesh.centre[e]
        hx, hy = mesh.h
        x[e, 0] = -cy
        x[e, 2] = -hy / 2 / np.sqrt(3)           # u_1 mode (0, 1): y-linear
        x[e, s + 0] = cx
        x[e, s + 1] = hx / 2 / np.sqrt(3)        # u_2 mode (1, 0): x-linear
    r = lev.A @ x.ravel()
    assert np.linalg.norm(r) <= 1e-12 * abs(lev.A).max() * np.linalg.norm(x)


def _block_counts(lev):
    """Number of nonzero s x s coupling sub-blocks per interior element."""
    A = lev.A.tocsr()
    s, nb = lev.s, lev.nb
    d = lev.mesh.d
    e = int(np.ravel_multi_index(tuple([2] * d), lev.mesh.n[::-1]))  # an interior element
    rows = A[e * nb:(e + 1) * nb, :].tocoo()
    keys = set()
    for r, c, v in zip(rows.row, rows.col, rows.data):
        if abs(v) > 1e-14 * abs(A).max() and c // nb != e:
            keys.add((c // nb, r // s, (c % nb) // s))
    return len(keys)


@pytest.mark.parametrize("d,gamma,expect", [(2, 0, 16), (2, 1, 22), (3, 0, 30), (3, 1, 48)])
def test_coupling_sub_block_count(d, gamma, expect):
    """Sparsity of the element coupling implied by the one-sided fluxes:
    2d(d+2) sub-blocks (standard) or 2d(2d+1) + d(d-1) (viscous stress)."""
    prob = P.generic(d, 6 if d == 2 else 5, 1, gamma, [P.PERIODIC] * (2 * d))
    lev = hierarchy.build_hierarchy(prob, max_levels=1)[0][0]
    assert _block_counts(lev) == expect


@pytest.mark.parametrize("gamma,d", [(0, 2), (1, 2), (1, 3)])
def test_parity_colouring_separates_couplings(gamma, d):
    prob = P.generic(d, 4, 1, gamma, [P.PERIODIC] * (2 * d))
    lev = hierarchy.build_hierarchy(prob, max_levels=1)[0][0]
    col = lev.mesh.colour()
    coo = lev.A.tocoo()
    ei, ej = coo.row // lev.nb, coo.col // lev.nb
    off = ei != ej
    assert not np.any(col[ei[off]] == col[ej[off]])


@pytest.mark.parametrize("prob", [
    P.generic(2, 8, 2, 0, [P.DIRICHLET, P.DIRICHLET, P.STRESS, P.DIRICHLET]),
    P.generic(2, 8, 3, 1, [P.DIRICHLET] * 3 + [P.STRESS]),
    P.generic(2, 8, 2, 1, [P.PERIODIC] * 4),
    P.generic(3, 4, 1, 1, [P.PERIODIC, P.PERIODIC, P.DIRICHLET, P.DIRICHLET, P.STRESS, P.DIRICHLET]),
])
def test_coarsening_equals_direct_assembly(prob):
    """T8 (Appendix B): Algorithm 2 on the n mesh equals assembling the LDG
    operator directly on the n/2 mesh (constant mu, Cartesian)."""
    levels, _ = hierarchy.build_hierarchy(prob, max_levels=2)
    coarse = prob.with_(n=tuple(v // 2 for v in prob.n))
    direct = hierarchy.build_hierarchy(coarse, max_levels=1)[0][0]
    diff = abs(levels[1].A - direct.A).max()
    assert diff <= 1e-12 * abs(direct.A).max()


def test_unsteady_penalties_coarsen_geometrically():
    """Algorithm 3: E_mu (x2) and E_rho (x1/2) coarsen to their direct
    assembly on the coarse mesh; M_rho by Galerkin."""
    prob = P.unsteady_periodic_3d(n=4, p=1, re=3.0)
    fine = ldg.fine_operators(prob)
    mesh_c = ldg.Mesh(3, (2, 2, 2), prob.lo, prob.hi, prob.bc)
    I = hierarchy.injection(fine["mesh"], mesh_c, prob.p)
    co = hierarchy.coarsen(fine, I, mesh_c, True)
    direct = ldg.fine_operators(prob.with_(n=(2, 2, 2)))
    for key in ("Emu", "Erho", "Mrho", "Mmu"):
        assert abs(co[key] - direct[key]).max() <= 1e-12 * abs(direct[key]).max(), key


def test_mass_coarsening_and_injection():
    """T9: M_2h = I^T M_h I equals the coarse mass matrix |E_c| I."""
    prob = P.generic(2, 8, 3, 0, [P.PERIODIC] * 4)
    ops = ldg.fine_operators(prob)
    mesh_c = ldg.Mesh(2, (4, 4), prob.lo, prob.hi, prob.bc)
    I = hierarchy.injection(ops["mesh"], mesh_c, prob.p)
    M2 = (I.T @ ops["M"] @ I).toarray()
    np.testing.assert_allclose(M2, mesh_c.vol * np.eye(M2.shape[0]), atol=1e-14)


def test_etimedep_reduces_to_harmonic_mean():
    """eq. (Etimedep): for proportional blocks x B and y B the combination is
    the harmonic combination xy/(x+y) B (the identity behind eq. Etimedep)."""
    s = 4
    rng = np.random.default_rng(3)
    B = rng.standard_normal((s, s))
    B = B @ B.T
    x, y = 0.7, 5.0
    Emu = sp.csr_matrix(x * B)
    Erho = sp.csr_matrix(y * B)
    E = hierarchy.combine_pressure_penalty(Emu, Erho, 1, s).toarray()
    np.testing.assert_allclose(E, x * y / (x + y) * B, rtol=1e-13)


def test_taugeneral_limits():
    """T11: eq. (taupgeneral) gives tau h / mu when rho = 0 and tau0 delta / (h rho)
    when mu = 0.  Checked on assembled E of a one-face problem."""
    base = P.unsteady_periodic_3d(n=2, p=1, re=1.0)
    tiny = 1e-300
    steady_like = base.with_(rho=lambda x: np.full(x.shape[:-1], tiny))
    inviscid = base.with_(mu=lambda x: np.full(x.shape[:-1], tiny))
    ref_mu = ldg.fine_operators(steady_like)
    ref_rho = ldg.fine_operators(inviscid)
    np.testing.assert_allclose(ref_mu["E"].toarray(), ref_mu["Emu"].toarray(), rtol=1e-12, atol=0)
    np.testing.assert_allclose(ref_rho["E"].toarray(), ref_rho["Erho"].toarray(), rtol=1e-12, atol=0)


# ------------------------------------------------- accuracy and solvers ----

def _l2_errors(prob, mg, x):
    lev = mg.levels[0]
    mesh, d, p, s = lev.mesh, prob.d, prob.p, lev.s
    q = p + 3
    xv, wv = mesh.volume_points(q)
    Phi = basis.tensor_basis(d, p, q)
    jac = mesh.vol / 2 ** d
    vals = np.einsum("qa,eva->eqv", Phi, x.reshape(mesh.ne, d + 1, s))
    ue, pe = prob.exact.u(xv), prob.exact.p(xv)
    out = []
    for v in range(d + 1):
        err = vals[..., v] - (ue[..., v] if v < d else pe)
        if all(b == P.PERIODIC for b in prob.bc) or (v == d and P.STRESS not in prob.bc):
            err = err - (err * wv).sum() / (wv.sum() * mesh.ne)   # kernel mode (constant)
        out.append(np.sqrt(jac * (err ** 2 * wv).sum()))
    return np.array(out)


def _solve_manufactured(prob):
    mg = multigrid.Multigrid(prob)
    b = mg.levels[0].P @ ldg.rhs(prob, mg.levels[0].ops)
    x, hist = mg.solve(b, rtol=1e-12, maxit=300)
    assert hist[-1] <= 1e-12
    return _l2_errors(prob, mg, x)


def test_order_periodic_standard():
    """Section 5.1: u and p converge at order p+1 (p = 2) with periodic conditions."""
    e8 = _solve_manufactured(P.periodic_standard_2d(n=8, p=2))
    e16 = _solve_manufactured(P.periodic_standard_2d(n=16, p=2))
    rate = np.log2(e8 / e16)
    assert np.all(np.abs(rate - 3.0) < 0.3), rate


def test_order_stress_variable_viscosity():
    """Sections 5.3-5.4: viscous-stress form, variable mu, Dirichlet + stress
    sides: u order p+1, p order about p+1/2 in L2 (p = 2)."""
    e8 = _solve_manufactured(P.stress_variable_mu_2d(n=8, p=2))
    e16 = _solve_manufactured(P.stress_variable_mu_2d(n=16, p=2))
    rate = np.log2(e8 / e16)
    assert np.all(np.abs(rate[:2] - 3.0) < 0.3), rate
    assert 2.0 < rate[2] < 3.2, rate


@pytest.mark.parametrize("prob", [
    P.periodic_standard_2d(n=4, p=1),
    P.generic(2, 4, 2, 0, [P.DIRICHLET] * 4),
    P.generic(2, 4, 3, 1, [P.DIRICHLET] * 3 + [P.STRESS]),
    P.generic(2, 4, 2, 1, [P.STRESS] * 4),
])
def test_vcycle_solve_matches_dense_pseudo_inverse(prob):
    """The converged V-cycle iteration equals the least-squares solution of a
    dense eigendecomposition, modulo the kernel."""
    mg = multigrid.Multigrid(prob)
    A = mg.A.toarray()
    lam, V = np.linalg.eigh(A)
    keep = np.abs(lam) > 1e-10 * np.abs(lam).max()
    rng = np.random.default_rng(7)
    b = rng.standard_normal(A.shape[0])
    b -= V[:, ~keep] @ (V[:, ~keep].T @ b)
    pinv = lambda v: V[:, keep] @ ((V[:, keep].T @ v) / lam[keep])
    x_ref = pinv(b)
    for _ in range(3):                      # refine the dense solution in FP64
        x_ref += pinv(b - A @ x_ref)
    x, hist = mg.solve(b, rtol=1e-13, maxit=400)
    x -= V[:, ~keep] @ (V[:, ~keep].T @ x)
    # Both are least-squares solutions up to their residuals:
    # ||x - x_ref|| <= (||b - A x|| + ||b - A x_ref||) / min |lambda|.
    bound = (np.linalg.norm(b - A @ x) + np.linalg.norm(b - A @ x_ref)) / np.abs(lam[keep]).min()
    assert np.linalg.norm(x - x_ref) <= 1.5 * bound + 1e-14 * np.linalg.norm(x_ref)
    assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


def test_colour_step_matches_block_definition():
    """One colour step equals x_i = A_ii^{-1}(b_i - sum_{j != i} A_ij x_j) from
    the dense operator, for every element of that colour."""
    prob = P.generic(2, 4, 2, 1, [P.DIRICHLET] * 3 + [P.STRESS])
    mg = multigrid.Multigrid(prob)
    sm = mg.sm[0]
    A = mg.A.toarray()
    nb = sm.nb
    rng = np.random.default_rng(1)
    x = rng.standard_normal(A.shape[0])
    b = rng.standard_normal(A.shape[0])
    for c in range(sm.ncol):
        ref = x.copy()
        for i in sm.elems[c]:
            sl = slice(i * nb, (i + 1) * nb)
            g = b[sl] - A[sl, :] @ x + A[sl, sl] @ x[sl]
            ref[sl] = np.linalg.solve(A[sl, sl], g)
        sm.colour_step(x, b, c)
        np.testing.assert_allclose(x, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_lexicographic_reference_converges():
    prob = P.periodic_standard_2d(n=8, p=2)
    mg = multigrid.Multigrid(prob)
    b = mg.levels[0].P @ ldg.rhs(prob, mg.levels[0].ops)
    x, hist = mg.solve(b, rtol=1e-10, maxit=60, lexicographic=True)
    assert hist[-1] <= 1e-10


def test_bottom_snaps_kernel():
    """The bottom solver snaps exactly the trivial kernel (T2 on the coarsest level)."""
    mg = multigrid.Multigrid(P.periodic_standard_2d(n=8, p=2))
    assert mg.kernel_dim_bottom == 3
    mg = multigrid.Multigrid(P.generic(2, 8, 2, 1, [P.DIRICHLET] * 3 + [P.STRESS]))
    assert mg.kernel_dim_bottom == 0


# ------------------------------------------------------- tau and rho pins ----

def test_golden_tables_match_problem_defaults():
    for form, d, p, tau in read_golden("table1_optimal_tau.txt"):
        assert P.TABLE1_TAU[(int(form), int(d), int(p))] == float(tau)
    for form, d, p, lo, hi in read_golden("table2_tau_window.txt"):
        assert P.TABLE2_WINDOW[(int(form), int(d), int(p))] == (float(lo), float(hi))


def _rho(prob, seed=1):
    mg = multigrid.Multigrid(prob)
    x0 = P.random_vector(prob.n_elements, prob.nb, seed=seed).ravel()
    return mg.gmres_rho(x0)


def test_rho_at_optimal_tau_and_breakdown():
    """Sections 4-5: with tau from Table 1 and V(3,3)-preconditioned GMRES,
    rho is within the typical 0.05-0.1 range; for tau = 1e-3 (below the 1e-2
    threshold) the V-cycle breaks down and rho approaches one."""
    golden = {r[0]: float(r[1]) for r in read_golden("convergence_statements.txt")}
    rho, it = _rho(P.periodic_standard_2d(n=16, p=2, nu=(3, 3)))
    assert rho <= golden["rho_typical_hi"], rho
    rho_bad, _ = _rho(P.periodic_standard_2d(n=16, p=2, nu=(3, 3), tau=1e-3))
    assert rho_bad >= 0.8, rho_bad


@pytest.mark.slow
def test_table1_tau_within_table2_window_of_oracle_minimum():
    """Table 1 / Table 2: the paper's optimal tau lies inside the 12.5 percent
    window of the oracle's own rho(tau) curve (viscous-stress form, p = 2)."""
    taus = [0.02, 0.03, 0.04, 0.05, 0.07, 0.1, 0.15]
    rhos = [_rho(P.generic(2, 32, 2, 1, [P.PERIODIC] * 4, tau=t, nu=(3, 3)))[0] for t in taus]
    rmin = min(rhos)
    rho_tab, _ = _rho(P.generic(2, 32, 2, 1, [P.PERIODIC] * 4, tau=P.TABLE1_TAU[(1, 2, 2)], nu=(3, 3)))
    assert rho_tab <= rmin ** (1 - 1 / 9), (rho_tab, rmin)
    lo, hi = P.TABLE2_WINDOW[(1, 2, 2)]
    best = taus[int(np.argmin(rhos))]
    assert lo * 0.8 <= best <= hi * 1.25, best


def test_bf16_rounding_is_round_to_nearest_even():
    v = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -3.140625])
    np.testing.assert_array_equal(multigrid.round_bf16(v), [1.0, 1.0 + 2 * 2.0 ** -7, 1.0, -3.140625])


def test_fp16_scaled_rounding_values():
    """Scaled FP16 storage: hand-computed values.  [1, 3, 1e-3]: max 3 =
    0.75 * 2^2, so the group is multiplied by 2^13; 8.192 rounds to 1049 * 2^-7
    (FP16 spacing 2^-7 on [8, 16)).  1 + 2^-11 is scaled by 2^14 to 16392, a tie
    between 16384 and 16400 (spacing 16), which goes to the even 16384.  A
    member 2^-41 below the maximum falls under half the smallest subnormal and
    becomes 0."""
    got = multigrid.round_fp16_scaled(np.array([[1.0, 3.0, 1e-3]]), axis=1)
    np.testing.assert_array_equal(got, [[1.0, 3.0, 1049 * 2.0 ** -7 / 2.0 ** 13]])
    np.testing.assert_array_equal(multigrid.round_fp16_scaled(np.array([1.0 + 2.0 ** -11]), axis=0), [1.0])
    np.testing.assert_array_equal(multigrid.round_fp16_scaled(np.array([1.0, 2.0 ** -41]), axis=0), [1.0, 0.0])
    np.testing.assert_array_equal(multigrid.round_fp16_scaled(np.zeros((2, 3)), axis=1), np.zeros((2, 3)))


def test_fp16_scaled_rounding_error_bound_and_groups():
    """Each entry is off by at most half an FP16 unit of its scaled value
    (relative 2^-11 for normal scaled values, absolute 2^-25 of the scale
    below), the groups are independent, and the sparse sub-block version
    equals the dense one applied per s x s sub-block."""
    rng = np.random.default_rng(0)
    a = rng.standard_normal((5, 6, 7)) * np.exp2(rng.integers(-30, 30, (5, 6, 1)))
    r = multigrid.round_fp16_scaled(a, axis=2)
    mx = np.abs(a).max(axis=2, keepdims=True)
    _, e = np.frexp(mx)
    scaled = np.abs(a) * np.exp2(15.0 - e)
    tol = np.where(scaled >= 2.0 ** -14, scaled * 2.0 ** -11, 2.0 ** -25) * np.exp2(e - 15.0)
    assert np.all(np.abs(r - a) <= tol)
    # rows are independent: rounding one row alone gives the same values
    np.testing.assert_array_equal(multigrid.round_fp16_scaled(a[2:3, 4:5], axis=2), r[2:3, 4:5])
    s, nbk = 3, 4
    A = sp.random(nbk * s, nbk * s, density=0.5, random_state=1, format="csr")
    A.data *= np.exp2(rng.integers(-20, 20, A.nnz))
    Rs = multigrid.round_fp16_subblocks(A, s).toarray()
    D = A.toarray().reshape(nbk, s, nbk, s)
    mxb = np.abs(D).max(axis=(1, 3), keepdims=True)
    _, eb = np.frexp(mxb)
    upb = np.exp2(15.0 - np.where(mxb > 0, eb, 0))
    ref = ((D * upb).astype(np.float16).astype(np.float64) / upb).reshape(nbk * s, nbk * s)
    np.testing.assert_array_equal(Rs, ref)


def test_bottom_solve_is_least_squares_solution():
    """The bottom solver returns the least-squares solution: orthogonal to the
    kernel, residual orthogonal to the range (Section 3 footnote)."""
    for prob in (P.periodic_standard_2d(n=8, p=2), P.generic(2, 8, 3, 1, [P.DIRICHLET] * 3 + [P.STRESS])):
        mg = multigrid.Multigrid(prob)
        A = mg.levels[-1].A.toarray()
        lam, V = np.linalg.eigh(A)
        ker = V[:, np.abs(lam) <= 1e-10 * np.abs(lam).max()]
        b = np.random.default_rng(2).standard_normal(A.shape[0])
        x = mg.bottom_solve(b)
        r = b - A @ x
        assert np.linalg.norm(ker.T @ x) <= 1e-12 * np.linalg.norm(x)
        assert np.linalg.norm(r - ker @ (ker.T @ r)) <= 1e-13 * np.linalg.norm(b)


def test_fgmres_matches_dense_solution_and_is_monotone():
    """Flexible GMRES with the V-cycle preconditioner: the residual never
    grows within a restart cycle, and the converged solution is the dense
    least-squares solution (bounded by both residuals)."""
    prob = P.generic(2, 8, 2, 1, [P.DIRICHLET] * 3 + [P.STRESS])
    mg = multigrid.Multigrid(prob)
    A = mg.A.toarray()
    b = np.random.default_rng(4).standard_normal(A.shape[0])
    x, hist = mg.fgmres(b, rtol=1e-12, maxit=100, restart=50)
    assert hist[-1] <= 1e-12
    assert all(h1 <= h0 * (1 + 1e-12) for h0, h1 in zip(hist[:-1], hist[1:]))
    lam = np.linalg.eigvalsh(A)
    x_ref = np.linalg.solve(A, b)
    bound = (np.linalg.norm(b - A @ x) + np.linalg.norm(b - A @ x_ref)) / np.abs(lam).min()
    assert np.linalg.norm(x - x_ref) <= 1.5 * bound + 1e-14 * np.linalg.norm(x_ref)


def test_learned_smoother_gradient_matches_finite_differences():
    """The oracle's back-propagated gradient of the MLP loss equals central
    finite differences of the loss (tiny network, FP64)."""
    from oracle import learned
    rng = np.random.default_rng(0)
    nin, hid, nout, rows = 7, 5, 3, 11
    F = rng.standard_normal((rows, nin))
    T = rng.standard_normal((rows, nout))
    w = 0.5 * rng.standard_normal(nin * hid + hid + hid * nout + nout)
    loss, g = learned.loss_and_grad(F, T, w, nin, hid, nout)
    eps = 1e-6
    fd = np.zeros_like(w)
    for i in range(w.size):
        wp, wm = w.copy(), w.copy()
        wp[i] += eps
        wm[i] -= eps
        fd[i] = (learned.loss_and_grad(F, T, wp, nin, hid, nout)[0] -
                 learned.loss_and_grad(F, T, wm, nin, hid, nout)[0]) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8)


def test_learned_features_neighbour_order():
    from oracle import learned
    mesh = ldg.Mesh(2, (4, 3), (0, 0), (1, 1), [P.DIRICHLET, P.DIRICHLET, P.PERIODIC, P.PERIODIC])
    nb = learned.face_neighbours(mesh)
    e = 1 + 4 * 0       # element (1, 0)
    assert list(nb[e]) == [0, 2, 1 + 4 * 2, 1 + 4 * 1]
    assert nb[0, 0] == -1 and nb[3, 1] == -1


def test_learned_residual_objective_gradient_matches_finite_differences():
    """Gradient of ||r - A delta(r)||^2 / ||r||^2 (the correction's training
    objective) against central finite differences on a 4x4, p=1 operator."""
    from oracle import learned
    prob = P.generic(2, 4, 1, 1, [P.DIRICHLET] * 3 + [P.STRESS])
    lev = hierarchy.build_hierarchy(prob, max_levels=1)[0][0]
    nbrs = learned.face_neighbours(lev.mesh)
    rng = np.random.default_rng(1)
    r = rng.standard_normal((lev.ne, lev.nb))
    nin, hid, nout = 5 * lev.nb, 6, lev.nb
    w = 0.1 * rng.standard_normal(nin * hid + hid + hid * nout + nout)
    loss, g = learned.residual_loss_and_grad(lev.A, r, nbrs, w, nin, hid, nout)
    eps = 1e-6
    idx = rng.choice(w.size, 40, replace=False)
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += eps
        wm[i] -= eps
        fd = (learned.residual_loss_and_grad(lev.A, r, nbrs, wp, nin, hid, nout)[0] -
              learned.residual_loss_and_grad(lev.A, r, nbrs, wm, nin, hid, nout)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-7 * np.abs(g).max()


# ------------------------------------------------------------ multi-phase ----

@pytest.mark.parametrize("ratio", [1e-6, 1e-3, 1e3, 1e6])
def test_multiphase_symmetry_kernel_and_colouring(ratio):
    """Section 5.6 square interface: symmetric operator (also after the sqrt(mu)
    scaling), periodic kernel of dimension d+1, and the greedy colouring
    separates every pair of coupled elements (interphase lifts couple
    elements two apart)."""
    prob = P.square_interface(n=8, p=1, mu_inner=ratio)
    levels, _ = hierarchy.build_hierarchy(prob)
    assert [l.ne for l in levels] == [64, 16]      # same-phase agglomeration stops at 4x4
    for lev in levels:
        A = lev.A
        assert abs(A - A.T).max() <= 1e-13 * abs(A).max()
        col = lev.mesh.colour()
        coo = A.tocoo()
        ei, ej = coo.row // lev.nb, coo.col // lev.nb
        off = (ei != ej) & (np.abs(coo.data) > 0)
        assert not np.any(col[ei[off]] == col[ej[off]])
    lam = np.linalg.eigvalsh(levels[0].A.toarray())
    assert int((np.abs(lam) <= 1e-10 * np.abs(lam).max()).sum()) == 3


def _mp_errors(prob, mg, x):
    lev = mg.levels[0]
    mesh, d, p, s = lev.mesh, prob.d, prob.p, lev.s
    q = p + 3
    xv, wv = mesh.volume_points(q)
    Phi = basis.tensor_basis(d, p, q)
    jac = mesh.vol / 2 ** d
    vals = np.einsum("qa,eva->eqv", Phi, x.reshape(mesh.ne, d + 1, s))
    ue, pe = prob.exact.u(xv), prob.exact.p(xv)
    out = []
    for v in range(d + 1):
        err = vals[..., v] - (ue[..., v] if v < d else pe)
        err = err - (err * wv).sum() / (wv.sum() * mesh.ne)
        out.append(np.sqrt(jac * (err ** 2 * wv).sum()))
    return np.array(out)


@pytest.mark.parametrize("ratio", [1e-6, 1e-3, 1e3, 1e6])
def test_multiphase_orders_and_rate(ratio):
    """Section 5.6: viscosity-upwinded fluxes with jump data and the sqrt(mu)
    scaling: velocity order p+1, pressure about p+1/2 (p = 2), and
    V(3,3)-preconditioned GMRES needs 7-10 iterations per 1e8 (rho <= 0.16)."""
    errs = []
    for n in (8, 16):
        prob = P.square_interface(n=n, p=2, mu_inner=ratio, nu=(3, 3))
        mg = multigrid.Multigrid(prob)
        b = mg.scale_rhs(mg.levels[0].P @ ldg.rhs(prob, mg.levels[0].ops))
        x, hist = mg.fgmres(b, rtol=1e-12, maxit=60, restart=60)
        assert hist[-1] <= 1e-12
        errs.append(_mp_errors(prob, mg, mg.unscale(x)))
    rate = np.log2(errs[0] / errs[1])
    assert np.all(rate[:2] > 2.7), rate
    assert rate[2] > 1.9, rate
    rho, it = mg.gmres_rho(P.random_vector(prob.n_elements, prob.nb, seed=1).ravel())
    assert rho <= 0.16, rho


# ------------------------------------------------------------ cycle shapes ----

@pytest.mark.parametrize("shape", [(2, 1, 64), (3, 1, 64), (1, 2, 64), (1, 2, 5), (2, 3, 7)])
def test_cycle_shape_visit_and_sweep_counts(shape):
    """W-cycles and variable V-cycles (Section 6) in closed form: level l < L-1
    is visited gamma^l times and smooths min(nu growth^l, max(nu, cap)) times
    before and after the coarse correction on every visit; the exactly solved
    bottom is entered once per visit of level L-2, gamma^(L-2) times."""
    gamma, growth, cap = shape
    prob = P.generic(2, 16, 1, 0, [P.DIRICHLET] * 3 + [P.STRESS], nu=(2, 1))
    mg = multigrid.Multigrid(prob, shape=shape)
    L = len(mg.levels)
    assert L == 4
    counts = [0] * (L - 1)
    bottoms = [0]
    for l, sm in enumerate(mg.sm):
        def counted(x, b, l=l, f=sm.sweep):
            counts[l] += 1
            return f(x, b)
        sm.sweep = counted
    solve = mg.bottom_solve

    def counted_bottom(b):
        bottoms[0] += 1
        return solve(b)
    mg.bottom_solve = counted_bottom
    b = np.random.default_rng(0).standard_normal(mg.A.shape[0])
    mg.vcycle(np.zeros_like(b), b)
    for l in range(L - 1):
        per_visit = sum(min(nu * growth ** l, max(nu, cap)) for nu in (2, 1))
        assert counts[l] == gamma ** l * per_visit, (l, counts)
    assert bottoms[0] == gamma ** (L - 2)


def test_w_cycle_limit_is_two_grid_cycle():
    """With many coarse visits the W-cycle's coarse correction converges to
    the exact coarse solution, so one cycle equals the two-grid cycle
    S^nu2 (x + I A_1^{-1} I^T (b - A S^nu1 x)) with a dense solve on level 1
    (kernel-free boundary conditions, three levels)."""
    prob = P.generic(2, 8, 2, 0, [P.DIRICHLET] * 3 + [P.STRESS], nu=(2, 2))
    mg = multigrid.Multigrid(prob, shape=(30, 1, 64))
    assert len(mg.levels) == 3
    rng = np.random.default_rng(3)
    b = rng.standard_normal(mg.A.shape[0])
    x0 = rng.standard_normal(mg.A.shape[0])
    xw = mg.vcycle(x0.copy(), b)
    x = x0.copy()
    for _ in range(2):
        mg.sm[0].sweep(x, b)
    rc = mg.I[0].T @ (b - mg.A @ x)
    x += mg.I[0] @ np.linalg.solve(mg.levels[1].A.toarray(), rc)
    for _ in range(2):
        mg.sm[0].sweep(x, b)
    assert np.linalg.norm(xw - x) <= 1e-12 * np.linalg.norm(x)
    # and a V-cycle is not that limit
    xv = multigrid.Multigrid(prob).vcycle(x0.copy(), b)
    assert np.linalg.norm(xv - x) >= 1e-4 * np.linalg.norm(x)


def test_variable_v_cycle_limit_is_two_grid_cycle():
    """A variable V-cycle whose smoothing on level 1 grows without bound (200
    sweeps per phase there) solves the level-1 problem exactly, so one cycle
    equals the same two-grid cycle with a dense coarse solve (three levels,
    kernel-free boundary conditions); the finest level keeps nu = 2."""
    prob = P.generic(2, 8, 2, 0, [P.DIRICHLET] * 3 + [P.STRESS], nu=(2, 2))
    mg = multigrid.Multigrid(prob, shape=(1, 100, 400))
    assert mg.sweeps(2, 0) == 2 and mg.sweeps(2, 1) == 200
    rng = np.random.default_rng(3)
    b = rng.standard_normal(mg.A.shape[0])
    x0 = rng.standard_normal(mg.A.shape[0])
    xv = mg.vcycle(x0.copy(), b)
    x = x0.copy()
    for _ in range(2):
        mg.sm[0].sweep(x, b)
    rc = mg.I[0].T @ (b - mg.A @ x)
    x += mg.I[0] @ np.linalg.solve(mg.levels[1].A.toarray(), rc)
    for _ in range(2):
        mg.sm[0].sweep(x, b)
    assert np.linalg.norm(xv - x) <= 1e-12 * np.linalg.norm(x)


def test_w_cycle_contracts_faster_than_v_cycle():
    """More coarse-grid work per cycle (W, or the variable V-cycle) gives a
    smaller rho of eq. (rho) than V(1,1) on the viscous-stress problem with
    mixed boundary conditions (Section 6 names both as candidates)."""
    prob = P.generic(2, 16, 2, 1, [P.DIRICHLET] * 3 + [P.STRESS], nu=(1, 1))
    x0 = P.random_vector(prob.n_elements, prob.nb, seed=1).ravel()
    rho_v, _ = multigrid.Multigrid(prob).gmres_rho(x0)
    rho_w, _ = multigrid.Multigrid(prob, shape=(2, 1, 64)).gmres_rho(x0)
    rho_vv, _ = multigrid.Multigrid(prob, shape=(1, 2, 64)).gmres_rho(x0)
    assert rho_w < 0.9 * rho_v and rho_vv < 0.9 * rho_v, (rho_v, rho_w, rho_vv)


def test_gmres_rho_history_and_spectrum_estimate():
    """Left-preconditioned GMRES of eq. (rho): every recorded residual equals
    the least-squares minimum min_y ||beta e1 - H_k y|| recomputed by numpy
    from the Arnoldi matrix; rho^n equals the final reduction; and the Ritz
    values of H_n (Section 4's GMRES estimate of the spectrum of V A) cluster
    tightly around 1 at Table 1's tau and spread for tau well above it."""
    spread = {}
    for tau in (None, 1.0):
        prob = P.periodic_standard_2d(n=16, p=2, nu=(3, 3), tau=tau)
        mg = multigrid.Multigrid(prob)
        x0 = P.random_vector(prob.n_elements, prob.nb, seed=1).ravel()
        rho, n, hist, H = mg.gmres_rho(x0, details=True)
        assert np.allclose(np.triu(H[: n + 1, :n], -1), H[: n + 1, :n])       # upper Hessenberg
        e1 = np.zeros(n + 1)
        e1[0] = 1.0
        for k in range(1, n + 1):
            y = np.linalg.lstsq(H[: k + 1, :k], e1[: k + 1], rcond=None)[0]
            assert abs(np.linalg.norm(e1[: k + 1] - H[: k + 1, :k] @ y) - hist[k]) <= 1e-10 * hist[k]
        assert hist[n] <= 1e-8 < hist[n - 1]
        assert abs(rho ** n - hist[n]) <= 1e-12 * hist[n]
        spread[tau] = np.abs(np.linalg.eigvals(H[:n, :n]) - 1.0).max()
    assert spread[None] <= 0.25 and spread[1.0] >= 2 * spread[None], spread


@pytest.mark.parametrize("prob", [
    P.generic(2, 8, 2, 0, [P.PERIODIC] * 4),
    P.generic(2, 8, 1, 0, [P.DIRICHLET, P.STRESS, P.DIRICHLET, P.DIRICHLET]),
    P.generic(3, 4, 1, 0, [P.PERIODIC] * 6),
    P.unsteady_periodic_3d(n=4, p=1, re=10.0),
], ids=lambda q: q.name or str(q.bc))
def test_two_colours_separate_standard_form_couplings(prob):
    """The standard form (gamma = 0, single phase) couples face neighbours
    only, so the checkerboard (i_1 + ... + i_d) mod 2 is a valid colouring of
    the block GS on every smoothing level; for the viscous-stress form the
    edge couplings join elements of the same checkerboard colour."""
    levels, _ = hierarchy.build_hierarchy(prob)
    for lev in levels[:-1]:
        col = lev.mesh.colour_two()
        coo = lev.A.tocoo()
        ei, ej = coo.row // lev.nb, coo.col // lev.nb
        off = ei != ej
        assert not np.any(col[ei[off]] == col[ej[off]])
    vs = hierarchy.build_hierarchy(P.generic(2, 4, 1, 1, [P.PERIODIC] * 4), max_levels=1)[0][0]
    coo = vs.A.tocoo()
    ei, ej = coo.row // vs.nb, coo.col // vs.nb
    col = vs.mesh.colour_two()
    assert np.any((ei != ej) & (col[ei] == col[ej]))


def test_two_colour_gs_contracts_at_least_as_well():
    """Checkerboard block GS (two launches per sweep in any dimension) against
    the 2^d parity colours on the standard form: rho of eq. (rho) is no larger
    (0.060 vs 0.078 for periodic p=2, 16^2; 0.065 vs 0.077 for the periodic
    cube, p=2, 8^3)."""
    for prob in (P.periodic_standard_2d(n=16, p=2, nu=(3, 3)),
                 P.generic(2, 16, 2, 0, [P.DIRICHLET] * 4, nu=(3, 3))):
        x0 = P.random_vector(prob.n_elements, prob.nb, seed=1).ravel()
        mg = multigrid.Multigrid(prob)
        rho_par, _ = mg.gmres_rho(x0)
        rho_two, _ = multigrid.Multigrid(prob, levels=mg.levels, injections=mg.I, two_colours=True).gmres_rho(x0)
        assert mg.sm[0].ncol == 4
        assert rho_two <= 0.9 * rho_par, (rho_two, rho_par)


# ------------------------------------------------ unsteady and 3D pins ----

def _rho_var():
    """Variable density rho = 1 + 0.5 sin 2pi x sin 2pi y (sympy and numpy forms)."""
    import sympy as sp
    rho_expr = lambda xs: 1 + sp.Rational(1, 2) * sp.sin(2 * sp.pi * xs[0]) * sp.sin(2 * sp.pi * xs[1])
    rho_np = lambda x: 1.0 + 0.5 * np.sin(2 * np.pi * x[..., 0]) * np.sin(2 * np.pi * x[..., 1])
    return rho_expr, rho_np


@pytest.mark.parametrize("gamma", [0, 1])
def test_unsteady_delta_limits(gamma):
    """eq. (timedep2) against its two limits, on every level (Algorithm 3):
    as delta -> 0 the mass term dominates, delta A_uu -> M_rho, which for a
    constant rho is rho |E| I in an orthonormal basis (|E| = (2^l h)^d on
    level l); as delta -> infinity the operator tends to the steady one of
    Algorithm 2 (eq. taupgeneral tends to tau h / mu).  A wrong 1/delta or
    rho scale, or a wrong combination of E_mu and E_rho, fails one of them."""
    rho0 = 2.5
    bc = [P.DIRICHLET] * 3 + [P.STRESS]
    rho = lambda x: np.full(x.shape[:-1], rho0)
    steady = P.generic(2, 8, 2, gamma, bc)
    lev_s, _ = hierarchy.build_hierarchy(steady)
    small, _ = hierarchy.build_hierarchy(steady.with_(rho=rho, delta=1e-14))
    large, _ = hierarchy.build_hierarchy(steady.with_(rho=rho, delta=1e12))
    assert len(lev_s) == len(small) == len(large) >= 2
    s = (steady.p + 1) ** 2
    nb = 3 * s
    for l, (ls, lsm, llg) in enumerate(zip(lev_s, small, large)):
        h = 1.0 / ls.mesh.n[0]
        # delta -> 0: velocity diagonal blocks of delta A are rho h^2 I (the
        # viscous part contributes delta A_visc ~ 1e-14 x O(500))
        Ad = hierarchy.diag_blocks(lsm.A, lsm.ne, nb) * 1e-14
        for v in range(2):
            blk = Ad[:, v * s:(v + 1) * s, v * s:(v + 1) * s]
            np.testing.assert_allclose(blk, np.broadcast_to(rho0 * h * h * np.eye(s), blk.shape),
                                       rtol=0, atol=1e-9 * rho0 * h * h)
        # delta -> infinity: the steady operator
        diff = abs(llg.A - ls.A).max()
        assert diff <= 1e-9 * abs(ls.A).max(), (l, diff)


def _unsteady_manufactured(n, gamma):
    rho_expr, rho_np = _rho_var()
    delta = 0.05
    ex = P.paper_solution(2, gamma, rho_expr=rho_expr, delta=delta)
    return P.generic(2, n, 2, gamma, [P.DIRICHLET] * 3 + [P.STRESS], rho=rho_np, delta=delta, exact=ex)


@pytest.mark.parametrize("gamma", [0, 1])
def test_order_unsteady_mass_term(gamma):
    """eq. (timedep1) with a fixed delta = 0.05 and variable density
    rho = 1 + 0.5 sin 2pi x sin 2pi y, Dirichlet on three sides and a stress
    condition on the fourth (p = 2): the velocity converges at order p+1 and
    the pressure at about p+1/2, as in the steady case (Section 5).  The mass
    term rho/delta u is as large as the viscous term here, so a wrong M_rho,
    1/delta factor or right-hand-side mass term would stop the convergence."""
    e8 = _solve_manufactured(_unsteady_manufactured(8, gamma))
    e16 = _solve_manufactured(_unsteady_manufactured(16, gamma))
    rate = np.log2(e8 / e16)
    assert np.all(np.abs(rate[:2] - 3.0) < 0.3), rate
    assert 2.0 < rate[2] < 3.3, rate


@pytest.mark.parametrize("gamma", [0, 1])
def test_order_3d(gamma):
    """3D assembly (faces orthogonal to all three axes, edge couplings of the
    viscous-stress form, 3D boundary and stress data): the manufactured
    solution of Appendix C on the unit cube with Dirichlet on five sides and a
    stress condition on the top (p = 1) converges at order p+1 = 2 in the
    velocity and at least p+1/2 in the pressure."""
    def prob(n):
        return P.generic(3, n, 1, gamma, [P.DIRICHLET] * 5 + [P.STRESS], exact=P.paper_solution(3, gamma))
    e4 = _solve_manufactured(prob(4))
    e8 = _solve_manufactured(prob(8))
    rate = np.log2(e4 / e8)
    assert np.all(np.abs(rate[:3] - 2.0) < 0.35), rate
    assert 1.4 < rate[3] < 2.4, rate


def _learned_setup(n=8):
    from oracle import learned
    prob = P.stress_variable_mu_2d(n=n, p=2, nu=(3, 3))
    mg = multigrid.Multigrid(prob)
    mesh = mg.levels[0].mesh
    nbrs = learned.face_neighbours(mesh)
    nb = prob.nb
    nin, hid = (1 + 2 * prob.d) * nb, 16
    nparam = nin * hid + hid + hid * nb + nb
    b = mg.levels[0].P @ ldg.rhs(prob, mg.levels[0].ops)
    return learned, prob, mg, nbrs, nin, hid, nb, nparam, b


def test_learned_solve_with_zero_correction_is_plain_refinement():
    """With all weights zero the correction is zero: every judged iteration
    then contracts exactly like the plain one, the iterates and the residual
    history are those of plain iterative refinement, whatever is decided."""
    learned, prob, mg, nbrs, nin, hid, nb, nparam, b = _learned_setup()
    x, hist, dec, ratios, kappa = learned.solve_with_correction(mg, b, np.zeros(nparam), nin, hid, nb, nbrs,
                                                                rtol=1e-10, maxit=60)
    x_ref, hist_ref = mg.solve(b, rtol=1e-10, maxit=60)
    assert len(hist) == len(hist_ref)
    np.testing.assert_allclose(hist, hist_ref, rtol=1e-12, atol=0)
    np.testing.assert_allclose(x, x_ref, rtol=0, atol=1e-12 * np.abs(x_ref).max())
    assert dec[:2] == [-1, -1] and abs(kappa - np.sqrt(hist[2] / hist[0])) <= 1e-15


def test_learned_solve_rejects_harmful_correction_and_switches_off():
    """A correction that destroys the iterate (huge random output weights) is
    undone in the two judged iterations after the kappa measurement, then
    switched off: decisions [-1, -1, 0, 0, -1, ...] and exactly the plain
    refinement's residual history."""
    learned, prob, mg, nbrs, nin, hid, nb, nparam, b = _learned_setup()
    w = np.random.default_rng(4).standard_normal(nparam) * 100.0
    x, hist, dec, ratios, kappa = learned.solve_with_correction(mg, b, w, nin, hid, nb, nbrs, rtol=1e-10, maxit=60)
    x_ref, hist_ref = mg.solve(b, rtol=1e-10, maxit=60)
    assert dec[:4] == [-1, -1, 0, 0] and all(v == -1 for v in dec[4:])
    assert ratios[2] > 1 and ratios[3] > 1
    np.testing.assert_allclose(hist, hist_ref, rtol=1e-9, atol=0)


def test_learned_solve_keeps_an_exact_correction():
    """A correction that is the exact remaining error would end the solve:
    replacing the network by delta = A^+ r_c (a perfect post-smoother, used
    here to check the bookkeeping) is kept at the first judged iteration and
    the next residual is at rounding level."""
    learned, prob, mg, nbrs, nin, hid, nb, nparam, b = _learned_setup()
    A = mg.A.toarray()
    orig = learned.correction
    try:
        learned.correction = lambda mg_, c, r, *a: np.linalg.lstsq(A, mg_.cycle_residual(0, c, r), rcond=None)[0]
        x, hist, dec, ratios, kappa = learned.solve_with_correction(mg, b, np.zeros(nparam), nin, hid, nb, nbrs,
                                                                    rtol=1e-10, maxit=60)
    finally:
        learned.correction = orig
    assert dec == [-1, -1, 1] and hist[-1] <= 1e-10 and ratios[2] < 1e-3


# ---------------------------------------------------- element clustering ----

def _clusters_by_coordinates(mesh):
    """Cluster of every element from its grid coordinates alone."""
    ci = mesh.idx // 2
    ncx = mesh.n[0] // 2
    return ci[:, 0] + ncx * ci[:, 1]


@pytest.mark.parametrize("gamma,bc", [(1, [P.DIRICHLET] * 3 + [P.STRESS]), (0, [P.PERIODIC] * 4)])
def test_cluster_colour_step_matches_block_definition(gamma, bc):
    """One colour step of the cluster smoother updates every cluster C of that
    colour to A_CC^{-1}(b_C - sum_{D != C} A_CD x_D), with the clusters
    formed from the element coordinates and the blocks cut from the dense
    operator; elements of other colours are untouched."""
    prob = P.generic(2, 8, 1, gamma, bc)
    mg = multigrid.Multigrid(prob, clusters=True)
    assert mg.clusters
    sm = mg.sm[0]
    A = mg.A.toarray()
    nb = prob.nb
    cl = _clusters_by_coordinates(mg.levels[0].mesh)
    rng = np.random.default_rng(2)
    x0, b = rng.standard_normal(A.shape[0]), rng.standard_normal(A.shape[0])
    for c in range(sm.ncol):
        x = x0.copy()
        sm.colour_step(x, b, c)
        expect = x0.copy()
        for C in range(sm.ncl):
            if sm.colour[C] != c:
                continue
            rows = np.concatenate([np.arange(e * nb, (e + 1) * nb) for e in np.nonzero(cl == C)[0]])
            others = np.setdiff1d(np.arange(A.shape[0]), rows)
            g = b[rows] - A[np.ix_(rows, others)] @ x0[others]
            expect[rows] = np.linalg.solve(A[np.ix_(rows, rows)], g)
        np.testing.assert_allclose(x, expect, rtol=0, atol=1e-11 * np.abs(expect).max())


@pytest.mark.parametrize("gamma", [0, 1])
def test_cluster_colouring_separates_coupled_clusters(gamma):
    """No two clusters of one colour couple: the checkerboard of clusters for
    the standard form, the four parity colours for the viscous-stress form."""
    prob = P.generic(2, 8, 1, gamma, [P.PERIODIC] * 4)
    mg = multigrid.Multigrid(prob, clusters=True)
    sm = mg.sm[0]
    assert sm.ncol == (2 if gamma == 0 else 4)
    cl = _clusters_by_coordinates(mg.levels[0].mesh)
    coo = mg.A.tocoo()
    ci, cj = cl[coo.row // prob.nb], cl[coo.col // prob.nb]
    off = (ci != cj) & (np.abs(coo.data) > 0)
    assert not np.any(sm.colour[ci[off]] == sm.colour[cj[off]])


def test_clustering_contracts_faster_at_p1():
    """Larger blocks for p = 1 (Concluding Remarks): with 2 x 2 clusters on
    the finest level, V(1,1)-preconditioned GMRES contracts at most 0.85
    times as fast (rho) as with single elements, on both forms."""
    for prob in (P.generic(2, 16, 1, 1, [P.DIRICHLET] * 3 + [P.STRESS]), P.generic(2, 16, 1, 0, [P.PERIODIC] * 4)):
        x0 = P.random_vector(prob.n_elements, prob.nb, seed=1).ravel()
        two = prob.gamma == 0
        rho_e, _ = multigrid.Multigrid(prob, two_colours=two).gmres_rho(x0, maxit=100)
        rho_c, _ = multigrid.Multigrid(prob, two_colours=two, clusters=True).gmres_rho(x0, maxit=100)
        assert rho_c <= 0.85 * rho_e, (rho_c, rho_e)


def test_clustering_not_applied_where_colours_would_not_close():
    """A periodic axis with an odd number of clusters (n = 6) keeps element
    blocks: a two- or four-colouring of 3 clusters around a wrap is invalid."""
    mg = multigrid.Multigrid(P.generic(2, 6, 1, 1, [P.PERIODIC] * 4), clusters=True)
    assert not mg.clusters


def test_earlier_bottom_keeps_the_contraction():
    """An exact solve on a finer coarsest level can only help: stopping the
    hierarchy of the 32 x 32, p = 3 viscous-stress problem at 8 x 8 (three
    levels) instead of 2 x 2 (five) keeps rho of V(3,3)-preconditioned GMRES
    within 5 % (and not worse)."""
    prob = P.stress_variable_mu_2d(n=32, p=3, nu=(3, 3))
    x0 = P.random_vector(prob.n_elements, prob.nb, seed=1).ravel()
    full = multigrid.Multigrid(prob)
    short = multigrid.Multigrid(prob, max_levels=3)
    assert len(full.levels) == 5 and len(short.levels) == 3
    rho_f, _ = full.gmres_rho(x0, maxit=100)
    rho_s, _ = short.gmres_rho(x0, maxit=100)
    assert rho_s <= rho_f * 1.05, (rho_s, rho_f)


# ------------------------------------------ cut cells of an embedded circle ----

def _cut_mesh(n=16, q=8):
    from oracle import cutcell
    return cutcell, cutcell.CutMesh(cutcell.Circle((0.5, 0.5), 0.25), n, q=q)


def test_cut_cells_area_and_perimeter():
    """Quadrature by dimension reduction: the inside pieces (and uncut inside
    cells) integrate 1 to the disc's area pi r^2 and the interface rule to the
    circumference 2 pi r, to 1e-13; the two pieces of every cut cell fill it."""
    cutcell, m = _cut_mesh()
    r = 0.25
    area_in = sum(p["area"] for p in m.pieces if p["phase"] == 1)
    perim = sum(w.sum() for (_, w, _) in m.interface.values())
    assert abs(area_in - np.pi * r * r) <= 1e-13
    assert abs(perim - 2 * np.pi * r) <= 1e-13
    for (i, j) in m.interface:
        a = m.pieces[m.piece_of[(i, j, 1)]]["area"] + m.pieces[m.piece_of[(i, j, 2)]]["area"]
        assert abs(a - m.cell_area) <= 1e-15


def test_cut_cells_polynomial_moments_of_the_disc():
    """Second moments over the disc in closed form: int x^2 = pi r^2 (c_x^2 +
    r^2/4), int x y = pi r^2 c_x c_y, summed over the inside pieces."""
    cutcell, m = _cut_mesh(n=20, q=8)
    c, r = np.array([0.5, 0.5]), 0.25
    mx2 = sum((p["weights"] * p["points"][:, 0] ** 2).sum() for p in m.pieces if p["phase"] == 1)
    mxy = sum((p["weights"] * p["points"][:, 0] * p["points"][:, 1]).sum() for p in m.pieces if p["phase"] == 1)
    assert abs(mx2 - np.pi * r * r * (c[0] ** 2 + r * r / 4)) <= 1e-13
    assert abs(mxy - np.pi * r * r * c[0] * c[1]) <= 1e-13


def test_cut_cells_divergence_theorem_per_piece():
    """Volume, face and interface rules agree with each other piece by piece:
    int_P div F = int_{dP} F.n for F = (x^2 y, x y^3), with the piece's faces
    (their same-phase parts, outward normals) and its arc (normal out of the
    circle for the inside piece, into it for the outside piece)."""
    cutcell, m = _cut_mesh(n=12, q=8)
    F = lambda p: np.stack([p[:, 0] ** 2 * p[:, 1], p[:, 0] * p[:, 1] ** 3], axis=1)
    divF = lambda p: 2 * p[:, 0] * p[:, 1] + 3 * p[:, 0] * p[:, 1] ** 2
    for (i, j), (xif, wif, nif) in m.interface.items():
        clo = m.lo + m.h * np.array([i, j])
        for ph, sgn in ((1, 1.0), (2, -1.0)):
            P = m.pieces[m.piece_of[(i, j, ph)]]
            vol = (P["weights"] * divF(P["points"])).sum()
            flux = sgn * (wif * (F(xif) * nif).sum(axis=1)).sum()
            for axis in (0, 1):
                for side in (0, 1):
                    fixed = clo[axis] + side * m.h[axis]
                    o = 1 - axis
                    parts = cutcell.face_parts(m.circle, clo[o], clo[o] + m.h[o], axis, fixed, 8)
                    pts, w = parts[ph]
                    if len(w):
                        flux += (2 * side - 1) * (w * F(pts)[:, axis]).sum()
            assert abs(vol - flux) <= 1e-13, (i, j, ph, vol, flux)


def test_cut_cells_merging():
    """Pieces below a quarter of their cell join a same-phase piece across a
    face of their cell that is not small itself; every element is then at
    least a quarter of a cell; both phases keep elements on both sides."""
    cutcell, m = _cut_mesh(n=32, q=6)
    assert m.merged_into
    for k, t in m.merged_into.items():
        p, q_ = m.pieces[k], m.pieces[t]
        assert p["area"] < 0.25 * m.cell_area <= q_["area"]
        assert p["phase"] == q_["phase"]
        (i, j), (ii, jj) = p["cell"], q_["cell"]
        assert abs(i - ii) + abs(j - jj) == 1
    reps = set(m.element)
    assert all(m.element_area(rep) >= 0.25 * m.cell_area for rep in reps)
    assert {m.pieces[r]["phase"] for r in reps} == {1, 2}


class _CutData:
    """Manufactured data of a problems.CutProblem as cutldg.rhs takes it."""

    def __init__(self, prob):
        self.prob, self.e = prob, prob.exact

    def u(self, x, chi):
        return self.e.u(x, chi=chi)

    def f(self, x, chi):
        return self.prob.forcing(x, chi)[:, :2]

    def fdiv(self, x, chi):
        return self.e.fdiv(x, chi=chi)

    def stress(self, x, n, chi):
        return self.e.stress(x, n, chi=chi)


def _cut_solve(n, p, mu_phase, gamma, rho_phase=None, delta=None, inside_only=False, radius=0.25):
    """Assemble on the cut mesh of the circle (Dirichlet box), solve the
    manufactured two-phase problem (the constant pressure, the kernel, fixed by
    a multiplier) and return the relative L2 velocity errors, the operator's
    asymmetry and the solve's residual.  With rho_phase and delta the unsteady
    problem (eq. timedep1; forcing with rho/delta u)."""
    import scipy.sparse.linalg as spla
    from oracle import cutcell, cutldg
    prob = P.CutProblem(n=n, p=p, gamma=gamma, mu_phase=mu_phase, rho_phase=rho_phase, delta=delta, radius=radius,
                        inside_only=inside_only)
    c, r = np.array([0.5, 0.5]), radius
    mesh = cutcell.CutMesh(cutcell.Circle(c, r), n, q=2 * p + 2, inside_only=inside_only)
    ops = cutldg.operators(mesh, p, mu_phase, P.TABLE1_TAU[(gamma, 2, p)], rho_phase=rho_phase, delta=delta,
                           tau0=prob.tau0)
    A = hierarchy.stokes_operator(ops, gamma, delta)
    ex = prob.exact
    b = cutldg.rhs(ops, _CutData(prob), gamma)
    ne, s = ops["mesh"].ne, ops["s"]
    k = np.zeros(A.shape[0])
    k[2 * ne * s + np.arange(ne) * s] = 1.0
    Aa = sp.bmat([[A, sp.csr_matrix(k[:, None])], [sp.csr_matrix(k[None, :]), None]], format="csc")
    x = spla.spsolve(Aa, np.concatenate([b, [0.0]]))[:-1]
    els = ops["els"]
    err, nrm = np.zeros(2), np.zeros(2)
    for e in range(ne):
        for kk in els.pieces[e]:
            pc = mesh.pieces[kk]
            Phi, _ = els.phi(e, pc["points"])
            w = pc["weights"]
            ue = ex.u(pc["points"], chi=np.full(len(w), els.phase[e]))
            for i in range(2):
                uh = Phi @ x[i * ne * s + e * s: i * ne * s + (e + 1) * s]
                err[i] += (w * (uh - ue[:, i]) ** 2).sum()
                nrm[i] += (w * ue[:, i] ** 2).sum()
    return np.sqrt(err / nrm), abs(A - A.T).max() / abs(A).max(), np.linalg.norm(A @ x - b) / np.linalg.norm(b)


@pytest.mark.parametrize("gamma,mu_phase", [(1, [1.0, 1e3]), (1, [1e3, 1.0]), (0, [1.0, 10.0])])
def test_cut_cell_ldg_order(gamma, mu_phase):
    """Appendix A on the merged cut-cell elements of the embedded circle (bases
    on the elements' bounding boxes, dense element mass matrices, the circle's
    curved normal in the interphase lift, penalties and jump data): the
    operator is symmetric and the two-phase manufactured solution's velocity
    converges at order p+1 = 3 (n = 8 -> 16), the accuracy pin of the
    cut-cell path, for viscosity ratios 1e3 and 1e-3 and both forms."""
    e8, a8, r8 = _cut_solve(8, 2, mu_phase, gamma)
    e16, a16, r16 = _cut_solve(16, 2, mu_phase, gamma)
    assert max(a8, a16) <= 1e-12 and max(r8, r16) <= 1e-10
    rate = np.log2(e8 / e16)
    assert np.all(np.abs(rate - 3.0) < 0.3), rate


def test_cut_cell_ldg_order_p1():
    e16, _, _ = _cut_solve(16, 1, [1.0, 10.0], 1)
    e32, _, _ = _cut_solve(32, 1, [1.0, 10.0], 1)
    rate = np.log2(e16 / e32)
    assert np.all(np.abs(rate - 2.0) < 0.3), rate


def test_cut_cell_unsteady_order():
    """The unsteady cut-cell operator (eq. timedep2: rho/delta M per phase and
    the general pressure penalty of eq. taupgeneral on intraphase faces) keeps
    velocity order p+1 = 3 for density ratio 1e3 and viscosity ratio 1e3."""
    e8, a8, _ = _cut_solve(8, 2, [1e3, 1.0], 1, rho_phase=[1e3, 1.0], delta=0.05)
    e16, a16, _ = _cut_solve(16, 2, [1e3, 1.0], 1, rho_phase=[1e3, 1.0], delta=0.05)
    assert max(a8, a16) <= 1e-12
    rate = np.log2(e8 / e16)
    assert np.all(np.abs(rate - 3.0) < 0.35), rate


def _cut_hierarchy(n=8, p=2, mu_phase=(1.0, 10.0), **kw):
    from oracle import cutcell, cuthier
    mesh = cutcell.CutMesh(cutcell.Circle((0.5, 0.5), 0.25), n, q=2 * p + 2)
    levels, inj = cuthier.build(mesh, p, list(mu_phase), P.TABLE1_TAU[(1, 2, p)], 1, **kw)
    return mesh, levels, inj


def _box_phi(lev, e, x, p):
    from oracle import cutldg
    t = cutldg.CutElements.__new__(cutldg.CutElements)
    t.p, t.box_lo, t.box_hi = p, lev.box_lo, lev.box_hi
    return cutldg.CutElements.phi(t, e, x)[0]


def test_cut_injection_reproduces_coarse_functions():
    """Section 3's injection on the cut hierarchy: a coarse Q_p function,
    prolongated, equals the coarse function at every quadrature point of every
    fine element (all three variables); pins the box mapping, the basis order
    and the block orientation of I."""
    p = 2
    mesh, levels, inj = _cut_hierarchy(p=p)
    els = levels[0].ops["els"]
    rng = np.random.default_rng(4)
    f0, c0 = levels[0], levels[1]
    xc = rng.standard_normal(c0.ne * c0.nb)
    xf = inj[0] @ xc
    parent = {}
    for f in range(f0.ne):
        # the coarse element whose box holds the fine element's box
        cands = [c for c in range(c0.ne) if c0.phase[c] == els.phase[f]
                 and np.all(c0.box_lo[c] <= f0.box_lo[f] + 1e-15) and np.all(f0.box_hi[f] <= c0.box_hi[c] + 1e-15)]
        rows = inj[0][f * f0.nb:(f + 1) * f0.nb].nonzero()[1] // c0.nb
        parent[f] = int(rows[0])
        assert parent[f] in cands
    worst = 0.0
    for f in range(f0.ne):
        for k in els.pieces[f]:
            x = mesh.pieces[k]["points"]
            Pf = _box_phi(f0, f, x, p)
            Pc = _box_phi(c0, parent[f], x, p)
            for v in range(3):
                uf = Pf @ xf[f * f0.nb + v * f0.s:f * f0.nb + (v + 1) * f0.s]
                uc = Pc @ xc[parent[f] * c0.nb + v * c0.s:parent[f] * c0.nb + (v + 1) * c0.s]
                worst = max(worst, np.abs(uf - uc).max())
    assert worst <= 1e-11 * np.abs(xc).max(), worst


def test_cut_coarse_mass_is_the_coarse_elements_mass():
    """Algorithm 2's coarse mass matrix I^T M I equals the mass matrix of each
    coarse element assembled directly by quadrature over its domain (the union
    of its members' pieces) in its own box basis."""
    from oracle.hierarchy import diag_blocks
    p = 2
    mesh, levels, inj = _cut_hierarchy(p=p)
    els = levels[0].ops["els"]
    f0, c0 = levels[0], levels[1]
    M2 = diag_blocks(c0.ops["M"], c0.ne, c0.s)
    direct = np.zeros_like(M2)
    for f in range(f0.ne):
        c = int(inj[0][f * f0.nb:(f + 1) * f0.nb].nonzero()[1][0] // c0.nb)
        for k in els.pieces[f]:
            Pc = _box_phi(c0, c, mesh.pieces[k]["points"], p)
            direct[c] += Pc.T @ (mesh.pieces[k]["weights"][:, None] * Pc)
    assert np.abs(M2 - direct).max() <= 1e-12 * np.abs(direct).max()


def test_cut_colouring_separates_coupled_elements():
    """Every level's greedy colouring gives different colours to any two
    elements that a block of the level's operator couples (Section 3: each
    colour step updates uncoupled elements only)."""
    mesh, levels, inj = _cut_hierarchy(n=16, p=1)
    for lev in levels[:-1]:
        coo = lev.A.tocoo()
        i, j = coo.row // lev.nb, coo.col // lev.nb
        off = i != j
        assert np.all(lev.colour[i[off]] != lev.colour[j[off]])


def test_cut_vcycle_contracts_independently_of_h():
    """Algorithm 1 on the cut hierarchy converges: the asymptotic contraction
    of x <- x + V(0, b - A x) with V(3,3) is below 0.5 at n = 16 and 32 and does
    not grow with n; the constant pressure (divided by D) is the kernel up to
    the quadrature error of the curved pieces (the divergence theorem holds
    for the cut-cell rules only to that error), and the bottom level snaps
    exactly one eigenvalue."""
    import types
    from oracle import multigrid
    ratios = []
    for n in (16, 32):
        mesh, levels, inj = _cut_hierarchy(n=n, p=2, mu_phase=(1.0, 1e3), scale=True)
        lev = levels[0]
        z = np.zeros((lev.ne, lev.nb))
        z[:, 2 * lev.s] = 1.0
        z = z.ravel() / lev.D
        assert np.linalg.norm(lev.A @ z) <= 1e-7 * abs(lev.A).max() * np.linalg.norm(z)
        mg = multigrid.Multigrid(types.SimpleNamespace(nu1=3, nu2=3, gamma=1), levels=levels, injections=inj)
        assert mg.kernel_dim_bottom == 1
        rng = np.random.default_rng(1)
        b = lev.A @ rng.standard_normal(lev.A.shape[0])
        x = np.zeros_like(b)
        rs = []
        for _ in range(10):
            r = b - lev.A @ x
            rs.append(np.linalg.norm(r))
            x = x + mg.precondition(r)
        ratios.append(rs[-1] / rs[-2])
    assert max(ratios) < 0.5, ratios
    assert ratios[1] < ratios[0] * 1.3, ratios


@pytest.mark.parametrize("gamma", [0, 1])
def test_cut_disc_order(gamma):
    """Section 5's curved domain: Stokes in the disc of radius 0.45 (the inside
    pieces only; Dirichlet data on the circle through the lift -int u v n and
    the penalty c_bdry p mu / h with the circle's outward normal), mu = 1: the
    operator is symmetric and the manufactured velocity converges at order
    p+1 = 3 (n = 8 -> 16), both forms."""
    e8, a8, r8 = _cut_solve(8, 2, [1.0], gamma, inside_only=True, radius=0.45)
    e16, a16, r16 = _cut_solve(16, 2, [1.0], gamma, inside_only=True, radius=0.45)
    assert max(a8, a16) <= 1e-12 and max(r8, r16) <= 1e-10
    rate = np.log2(e8 / e16)
    assert np.all(np.abs(rate - 3.0) < 0.35), rate


def test_float32_cycle_emulation_tracks_the_fp64_cycle():
    """The oracle's float32 cycle (float32 vectors, products and sums; FP32
    injection; FP64 bottom) takes the same steps as its FP64-vector cycle with
    the same FP32-rounded blocks: the two agree to FP32 rounding amplified by
    the cycle (1e-5), and the float32 cycle is not the FP64 one (it differs by
    more than 1e-9)."""
    prob = P.stress_variable_mu_2d(n=8, p=2)
    mg = multigrid.Multigrid(prob, storage="fp32")
    b = np.random.default_rng(0).uniform(-1, 1, prob.n_dofs)
    x64 = mg.precondition(b)
    x32 = mg.precondition_fp32(b)
    d = np.linalg.norm(x32 - x64) / np.linalg.norm(x64)
    assert 1e-9 < d <= 1e-5, d


# ---- Chebyshev-accelerated block Gauss-Seidel (Concluding Remarks; oracle/chebyshev.py)

def _gs_pair(prob):
    mg = multigrid.Multigrid(prob, two_colours=prob.gamma == 0 and prob.phase is None)
    sm = mg.sm[0]
    A = mg.levels[0].A

    def minv(r):
        z = np.zeros_like(r)
        sm.sweep(z, r)
        return z
    return mg, sm, A, minv


def test_chebyshev_degree_one_is_a_gauss_seidel_sweep():
    """One step with theta = 1 is x + M^{-1}(b - A x): one coloured block
    Gauss-Seidel sweep, whatever delta^2."""
    from oracle import chebyshev
    mg, sm, A, minv = _gs_pair(P.stress_variable_mu_2d(n=4, p=2))
    rng = np.random.default_rng(41)
    x0, b = rng.uniform(-1, 1, A.shape[0]), rng.uniform(-1, 1, A.shape[0])
    ref = x0.copy()
    sm.sweep(ref, b)
    for d2 in (-0.3, 0.0, 0.2):
        x = chebyshev.chebyshev_iteration(lambda v: A @ v, minv, x0.copy(), b, 1, 1.0, d2)
        assert np.abs(x - ref).max() <= 1e-13 * np.abs(ref).max()


def test_chebyshev_error_is_the_scaled_chebyshev_polynomial():
    """Textbook property on a symmetric positive definite diagonal operator
    with spectrum in [a, b] and M = I: after k steps with theta = (a + b) / 2,
    delta = (b - a) / 2 each eigencomponent of the error is multiplied by
    T_k((theta - lambda) / delta) / T_k(theta / delta)."""
    from numpy.polynomial import chebyshev as C
    from oracle import chebyshev
    lam = np.linspace(0.2, 3.0, 40)
    a, b_ = lam.min(), lam.max()
    theta, delta = 0.5 * (a + b_), 0.5 * (b_ - a)
    xs = np.random.default_rng(43).uniform(-1, 1, lam.size)
    rhs = lam * xs
    for k in (1, 2, 3, 5, 8):
        x = chebyshev.chebyshev_iteration(lambda v: lam * v, lambda r: r, np.zeros_like(xs), rhs, k, theta,
                                          delta ** 2)
        Tk = np.zeros(k + 1)
        Tk[k] = 1.0
        factor = C.chebval((theta - lam) / delta, Tk) / C.chebval(theta / delta, Tk)
        assert np.abs((xs - x) - factor * xs).max() <= 1e-12


def test_chebyshev_real_recurrence_matches_complex_form():
    """With imaginary foci (delta^2 < 0) Saad's recurrence in complex
    arithmetic produces real iterates, equal to the real recurrence in
    delta^2: pins the rewriting q_k = rho_k / delta."""
    from oracle import chebyshev
    mg, sm, A, minv = _gs_pair(P.periodic_standard_2d(n=4, p=1))
    rng = np.random.default_rng(47)
    x0, b = rng.uniform(-1, 1, A.shape[0]), rng.uniform(-1, 1, A.shape[0])
    for theta, d2 in ((0.9, -0.2), (1.1, -0.05), (0.8, 0.1)):
        xr = chebyshev.chebyshev_iteration(lambda v: A @ v, minv, x0.copy(), b, 4, theta, d2)
        delta = np.sqrt(complex(d2))
        xc = chebyshev.chebyshev_complex(lambda v: A @ v, minv, x0.copy(), b, 4, theta, delta)
        scale = np.abs(xr).max()
        assert np.abs(xc.imag).max() <= 1e-12 * scale
        assert np.abs(xc.real - xr).max() <= 1e-12 * scale


def test_chebyshev_cycle_with_theta_one_and_zero_delta_is_the_plain_cycle():
    """theta = 1, delta^2 = 0 makes every step x + M^{-1}(b - A x): the
    Chebyshev V-cycle is Algorithm 1's V-cycle."""
    from oracle import chebyshev
    prob = P.stress_variable_mu_2d(n=8, p=2)
    mg = multigrid.Multigrid(prob)
    mc = chebyshev.ChebyshevMultigrid(prob, params=[(1.0, 0.0)] * len(mg.sm))
    r = np.random.default_rng(53).uniform(-1, 1, prob.n_dofs)
    xp, xc = mg.precondition(r), mc.precondition(r)
    assert np.abs(xp - xc).max() <= 1e-12 * np.abs(xp).max()


def test_chebyshev_does_not_beat_plain_sweeps_at_equal_passes():
    """Measured comparison behind the decision not to put the Chebyshev
    smoother on the GPU.  A Chebyshev phase of degree k costs k sweeps and
    k - 1 residuals, i.e. k + (k - 1) passes over the blocks when a residual
    pass is counted like a sweep; degree 2 costs the three passes of plain
    V(3,3)'s phase.  The best (theta, delta^2) of a grid over theta in
    [0.7, 1.1] and delta^2 in [-0.3, 0.2] (found on these 8 x 8, p = 2
    problems: (0.85, 0) viscous stress, (0.9, -0.1) periodic standard form)
    gives a V(2,2)-Chebyshev rho above plain V(3,3)'s."""
    from oracle import chebyshev
    for prob, best in ((P.stress_variable_mu_2d(n=8, p=2), (0.85, 0.0)),
                       (P.periodic_standard_2d(n=8, p=2), (0.9, -0.1))):
        two = prob.gamma == 0 and prob.phase is None
        x0 = np.random.default_rng(0).uniform(-1, 1, prob.n_dofs)
        plain = multigrid.Multigrid(prob.with_(nu1=3, nu2=3), two_colours=two).gmres_rho(x0)[0]
        p2 = prob.with_(nu1=2, nu2=2)
        mg2 = multigrid.Multigrid(p2, two_colours=two)
        cheb = chebyshev.ChebyshevMultigrid(p2, params=[best] * len(mg2.sm), two_colours=two).gmres_rho(x0,
                                                                                                     maxit=60)[0]
        assert cheb > plain, (cheb, plain)


# ---- 3D cut cells of an embedded sphere (Section 5's sphere; oracle/cutcell3d.py)

def _sphere_grid(S, n, q):
    from oracle import cutcell3d as C3
    h = 1.0 / n
    out = []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                lo = np.array([i, j, k]) * h
                hi = lo + h
                cl = C3.classify(S, lo, hi)
                if cl == 0:
                    out.append((lo, hi, 0, C3.cell_rules(S, lo, hi, q)))
                else:
                    out.append((lo, hi, cl, C3._box_rule(lo, hi, q)))
    return out


def test_sphere_cut_cells_volume_area_and_moment():
    """Ball volume 4/3 pi r^3, sphere area 4 pi r^2 and the second moment
    int_ball |x - c|^2 = 4 pi r^5 / 5, summed over the cut and uncut cells of
    a 10^3 grid (q = 6); the inside and outside rules together give the box."""
    from oracle import cutcell3d as C3
    S = C3.Sphere((0.51, 0.47, 0.53), 0.3)
    r = S.r
    vin = vtot = area = m2 = 0.0
    for lo, hi, cl, rules in _sphere_grid(S, 10, 6):
        if cl == 0:
            (xi, wi), (xo, wo), (xs, ws, ns) = rules
            vin += wi.sum()
            vtot += wi.sum() + wo.sum()
            area += ws.sum()
            m2 += (wi * ((xi - S.c) ** 2).sum(1)).sum()
        else:
            x, w = rules
            vtot += w.sum()
            if cl < 0:
                vin += w.sum()
                m2 += (w * ((x - S.c) ** 2).sum(1)).sum()
    assert abs(vin - 4.0 / 3.0 * np.pi * r ** 3) <= 1e-10
    assert abs(area - 4.0 * np.pi * r ** 2) <= 1e-8
    assert abs(m2 - 4.0 * np.pi * r ** 5 / 5.0) <= 1e-11
    assert abs(vtot - 1.0) <= 1e-13


def test_sphere_cut_cells_divergence_theorem_per_piece():
    """For a cubic vector field F, on the inside and the outside piece of every
    cut cell: int div F dV equals the flux through the piece's boundary (the
    sphere patch with its normal, pointing out of the ball, and the piece's
    parts of the six cell faces), to 1e-9 of the cell's scale."""
    from oracle import cutcell3d as C3
    S = C3.Sphere((0.49, 0.52, 0.5), 0.27)
    rng = np.random.default_rng(61)
    A = rng.uniform(-1, 1, (3, 4, 3))   # F_a = sum_m A[a, m, b] x_b^m

    def F(x):
        return np.stack([sum(A[a, m, b] * x[:, b] ** m for m in range(4) for b in range(3)) for a in range(3)], 1)

    def divF(x):
        return sum(sum(m * A[a, m, a] * x[:, a] ** (m - 1) for m in range(1, 4)) for a in range(3))
    q = 6
    checked = 0
    for lo, hi, cl, rules in _sphere_grid(S, 8, q):
        if cl != 0:
            continue
        (xi, wi), (xo, wo), (xs, ws, ns) = rules
        flux_s = (ws * (F(xs) * ns).sum(1)).sum()
        for ph, (x, w), sgn in ((1, (xi, wi), 1.0), (2, (xo, wo), -1.0)):
            flux = sgn * flux_s
            for axis in range(3):
                for value, out in ((lo[axis], -1.0), (hi[axis], 1.0)):
                    fx, fw = C3.face_parts(S, lo, hi, axis, value, q)[ph]
                    if len(fw):
                        flux += out * (fw * F(fx)[:, axis]).sum()
            vol = (w * divF(x)).sum()
            assert abs(vol - flux) <= 1e-9 * (hi[0] - lo[0]) ** 2, (lo, ph, vol, flux)
        checked += 1
    assert checked > 50


def test_sphere_inside_one_cell_is_handled_by_subdivision():
    """A sphere wholly inside one cell: every height direction has the
    silhouette crossing the cell's tangential rectangle, so the cell is split
    until one does not; the rules still give the ball's volume and the
    sphere's area."""
    from oracle import cutcell3d as C3
    S = C3.Sphere((0.4, 0.55, 0.45), 0.2)
    (xi, wi), (xo, wo), (xs, ws, ns) = C3.cell_rules(S, np.zeros(3), np.ones(3), 8)
    assert abs(wi.sum() - 4.0 / 3.0 * np.pi * 0.2 ** 3) <= 1e-11
    assert abs(ws.sum() - 4.0 * np.pi * 0.2 ** 2) <= 1e-9
    assert abs(wi.sum() + wo.sum() - 1.0) <= 1e-13
    assert np.abs(np.linalg.norm(xs - S.c, axis=1) - 0.2).max() <= 1e-14


def test_cut_cell_rules_converge_on_coarse_cells():
    """The 2D rules grade toward the circle's extreme points (square-root
    branch points of the chord and of ds / dt): on an 8 x 8 grid cut by the
    circle of radius 1/4 the disc area and the perimeter are exact to 1e-13 at
    q = 8, and a rectangle cut by a disc whose extreme point lies just beyond
    the rectangle (0.0013 of a cell width away) gets its area to 1e-13."""
    from oracle import cutcell
    m = cutcell.CutMesh(cutcell.Circle((0.5, 0.5), 0.25), 8, q=8)
    area = sum(p["area"] for p in m.pieces if p["phase"] == 1)
    perim = sum(w.sum() for (_, w, _) in m.interface.values())
    assert abs(area - np.pi / 16) <= 1e-13 and abs(perim - np.pi / 2) <= 1e-13
    c2, rho = np.array([0.52, 0.5]), np.sqrt(0.27 ** 2 - 0.24 ** 2)
    (x, w), _, _ = cutcell.cell_rules(cutcell.Circle(c2, rho), np.array([0.375, 0.375]), np.array([0.5, 0.5]), 8)
    # area of the rectangle [0.375, 0.5]^2 within the disc, by the circular-segment formula:
    # the disc part with y <= 0.5 minus the part with z < 0.375 (none: 0.5 - rho > 0.375)
    dy = 0.52 - 0.5
    half = rho * rho * np.arccos(dy / rho) - dy * np.sqrt(rho * rho - dy * dy)   # segment y <= 0.5
    assert abs(w.sum() - 0.5 * half) <= 1e-13


def test_sphere_cut_mesh_merging():
    """The 3D cut mesh of a sphere (8^3 cells): the pieces keep the ball's
    volume and the box's; after merging every element holds at least a
    quarter of a cell, has one phase, and every join links face neighbours
    that share a positive same-phase face area."""
    from oracle import cutcell3d as C3
    S = C3.Sphere((0.48, 0.53, 0.5), 0.29)
    m = C3.CutMesh3D(S, 8, q=6)
    vin = sum(p["volume"] for p in m.pieces if p["phase"] == 1)
    assert abs(vin - 4.0 / 3.0 * np.pi * S.r ** 3) <= 1e-10
    assert abs(sum(p["volume"] for p in m.pieces) - 1.0) <= 1e-12
    assert len(m.merged_into) > 0
    groups = {}
    for k, rep in enumerate(m.element):
        groups.setdefault(rep, []).append(k)
    for rep, members in groups.items():
        assert sum(m.pieces[k]["volume"] for k in members) >= 0.25 * m.cell_volume
        assert len({m.pieces[k]["phase"] for k in members}) == 1
    for k, tgt in m.merged_into.items():
        a, b = np.array(m.pieces[k]["cell"]), np.array(m.pieces[tgt]["cell"])
        assert np.abs(a - b).sum() == 1 and m.pieces[k]["phase"] == m.pieces[tgt]["phase"]
        axis = int(np.nonzero(b - a)[0][0])
        assert m.shared_face_area(tuple(a), axis, int((b - a)[axis]), m.pieces[k]["phase"]) > 0
