"""The bottom solver's pseudo-inverse on the host (Section 3 footnote:
least-squares solution with near-zero eigenvalues snapped), through the C
ABI without a device: against numpy's dense inverse / eigendecomposition on
random, rank-deficient and structured symmetric matrices, and on the
oracle's bottom operators of the test problems."""
import numpy as np
import pytest

from paper_1911_05888_gb300 import native, problems as P
from oracle import multigrid

pytestmark = pytest.mark.skipif(not __import__("os").path.exists(native.LIB_PATH), reason="library not built")


def _sym(n, seed):
    a = np.random.default_rng(seed).standard_normal((n, n))
    return a + a.T


@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 300])
def test_random_symmetric_equals_inverse(n):
    A = _sym(n, n)
    pinv, sn = native.host_pseudo_inverse(A)
    ref = np.linalg.inv(A)
    assert sn == 0
    assert np.linalg.norm(pinv - ref) <= 1e-14 * np.linalg.cond(A) * np.linalg.norm(ref)
    assert np.allclose(pinv, pinv.T, atol=1e-13 * np.abs(pinv).max())


@pytest.mark.parametrize("n,k", [(5, 1), (40, 3), (200, 17)])
def test_rank_deficient_snaps_kernel(n, k):
    rng = np.random.default_rng(n + k)
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = rng.uniform(0.5, 4.0, n) * rng.choice([-1.0, 1.0], n)
    lam[:k] = 0.0
    A = (U * lam) @ U.T
    pinv, sn = native.host_pseudo_inverse(A)
    inv = np.where(lam != 0, 1.0 / np.where(lam != 0, lam, 1.0), 0.0)
    ref = (U * inv) @ U.T
    assert sn == k
    assert np.linalg.norm(pinv - ref) <= 1e-12 * np.linalg.norm(ref)
    # Moore-Penrose conditions
    assert np.linalg.norm(A @ pinv @ A - A) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(pinv @ A @ pinv - pinv) <= 1e-12 * np.linalg.norm(pinv)


def test_structured_matrices():
    # diagonal with repeated entries, identity, zero, already tridiagonal,
    # a zero column in the middle (Householder with a zero vector)
    D = np.diag([3.0, 3.0, -2.0, 3.0, 0.0, 5.0])
    pinv, sn = native.host_pseudo_inverse(D)
    assert sn == 1
    np.testing.assert_allclose(np.diag(pinv), [1 / 3, 1 / 3, -1 / 2, 1 / 3, 0.0, 1 / 5], rtol=1e-15, atol=1e-300)
    # smallness is judged after equilibration (row scales removed): a tiny
    # but isolated diagonal entry is a genuine eigenvalue, inverted exactly
    pinv, sn = native.host_pseudo_inverse(np.diag([1.0, 1e-14, 2.0]))
    assert sn == 0 and abs(pinv[1, 1] * 1e-14 - 1) <= 1e-15
    pinv, sn = native.host_pseudo_inverse(np.eye(9))
    assert sn == 0 and np.allclose(pinv, np.eye(9), rtol=0, atol=1e-15)
    pinv, sn = native.host_pseudo_inverse(np.zeros((4, 4)))
    assert sn == 4 and not pinv.any()
    T = np.diag(np.full(30, 2.0)) - np.diag(np.ones(29), 1) - np.diag(np.ones(29), -1)
    pinv, sn = native.host_pseudo_inverse(T)
    assert sn == 0 and np.linalg.norm(pinv @ T - np.eye(30)) <= 1e-12
    Z = _sym(12, 5)
    Z[4, :] = 0.0
    Z[:, 4] = 0.0
    pinv, sn = native.host_pseudo_inverse(Z)
    assert sn == 1 and np.linalg.norm(Z @ pinv @ Z - Z) <= 1e-12 * np.linalg.norm(Z)


def test_invalid_arguments():
    with pytest.raises(native.StkError):
        native.host_pseudo_inverse(np.eye(3), theta=1.5)


@pytest.mark.parametrize("prob", [
    P.periodic_standard_2d(n=8, p=2),
    P.generic(2, 8, 2, 1, [P.DIRICHLET] * 3 + [P.STRESS]),
    P.generic(3, 4, 1, 1, [P.DIRICHLET, P.STRESS, P.PERIODIC, P.PERIODIC, P.DIRICHLET, P.DIRICHLET]),
    P.unsteady_periodic_3d(n=8, p=2, re=10.0),
    P.square_interface(n=8, p=3, mu_inner=1e3),
], ids=lambda q: q.name or str(q.bc))
def test_bottom_operators_match_oracle(prob):
    """The oracle's bottom operators (up to 864 unknowns): the same snapped
    count as the oracle's kernel dimension, and the least-squares solution of
    consistent and inconsistent right-hand sides within 1e-15 cond(A) of the
    oracle's (refined) one -- about ten unit roundoffs times the condition
    number over the nonzero eigenvalues, the forward error of a backward
    stable solve; observed 1e-14 to 4e-12."""
    mg = multigrid.Multigrid(prob)
    A = mg.levels[-1].A.toarray()
    pinv, sn = native.host_pseudo_inverse(A)
    assert sn == mg.kernel_dim_bottom
    lam = np.abs(np.linalg.eigvalsh(A))
    nz = lam > 1e-10 * lam.max()
    tol = 1e-15 * lam[nz].max() / lam[nz].min()
    rng = np.random.default_rng(3)
    for k in range(4):
        b = rng.standard_normal(A.shape[0])
        if k < 3:
            b = A @ b                                    # consistent
        x = pinv @ b
        xo = mg.bottom_solve(b)
        assert np.linalg.norm(x - xo) <= tol * np.linalg.norm(xo)
