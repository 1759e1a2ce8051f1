"""Pins of the oracle's V-cycle (Algorithm 1) and solve loop (no GPU)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from tests import dense_ref as D


def _cycle_matrix(mg, n):
    """Error propagation of one oracle V-cycle: b = 0, x0 = unit vectors."""
    E = np.zeros((n * n, n * n))
    zero = np.zeros((n, n))
    for c in range(n * n):
        e = np.zeros(n * n)
        e[c] = 1.0
        E[:, c] = mg.vcycle(zero, e.reshape(n, n)).ravel()
    return E


@pytest.mark.parametrize("coarsest,ns", [(7, [15, 7]), (3, [15, 7, 3])])
@pytest.mark.parametrize("eps,theta", [(1.0, 0.0), (0.01, math.pi / 6)])
def test_vcycle_equals_dense_recursion(coarsest, ns, eps, theta):
    """Two- and three-level V(1,1) with Jacobi: the oracle's cycle equals the dense recursion
    E = S (I - P (I - E_c) Ac^-1 P^T A) S built from Kronecker P and dense Galerkin products."""
    n = 15
    s = O.q1_rotated_stencil(eps, theta)
    mg = O.Multigrid(O.const_field(n, s), coarsest_n=coarsest)
    assert [mg.n(l) for l in range(mg.levels)] == ns
    E = _cycle_matrix(mg, n)
    Ed = D.vcycle_matrix(D.const_matrix(s, n), ns)
    np.testing.assert_allclose(E, Ed, atol=1e-12)


def test_restriction_scaling_with_its_galerkin_operator_is_immaterial():
    """Algorithm 1 restricts with P^T and coarsens with P^T A P; the paper's full-weighting
    stencil is P^T / 4.  Scaling the restriction and the coarse operator together leaves
    the cycle unchanged (Jacobi on a scaled operator is the same smoother); full weighting
    with P^T A P instead under-corrects by 4 and converges visibly slower."""
    n = 15
    s = O.q1_rotated_stencil(0.05, 0.6)
    mg = O.Multigrid(O.const_field(n, s), coarsest_n=3)
    E = _cycle_matrix(mg, n)
    A = D.const_matrix(s, n)
    np.testing.assert_allclose(D.vcycle_matrix(A, [15, 7, 3], rscale=0.25), E, atol=1e-12)
    Em = D.vcycle_matrix(A, [15, 7, 3], rscale=0.25, mixed=True)
    rho = lambda M: np.abs(np.linalg.eigvals(M)).max()
    assert np.abs(Em - E).max() > 1e-2 and rho(Em) > rho(E) + 0.1


def test_vcycle_with_per_point_kernels_equals_dense():
    """Same check with arbitrary per-point 3x3 smoothing kernels H (the CNN smoother form)
    on a variable-coefficient operator, with two pre- and one post-smoothing step."""
    n = 15
    rng = np.random.default_rng(7)
    st = O.varcoef5_field(n, np.exp(rng.standard_normal((n + 1, n + 1))))
    mg = O.Multigrid(st, coarsest_n=3, nu1=2, nu2=1)
    Ws = []
    for l in range(mg.levels - 1):
        nl = mg.n(l)
        W = O.jacobi_kernels(mg.field(l)) * (1 + 0.3 * rng.standard_normal((9, nl, nl)))
        W += 0.02 * rng.standard_normal((9, nl, nl)) / mg.field(l)[4]
        mg.set_kernels(l, W)
        Ws.append(W)
    E = _cycle_matrix(mg, n)
    Ed = D.vcycle_matrix(D.field_matrix(st), [15, 7, 3],
                         smoother=lambda l, Al: D.kernels_matrix(Ws[l]), nu1=2, nu2=1)
    np.testing.assert_allclose(E, Ed, atol=1e-11)


def test_asymptotic_factor_is_spectral_radius():
    """The oracle's cycle operator has the dense recursion's spectral radius (Arnoldi on
    the oracle's V-cycle as a linear operator), and repeated cycles converge at that rate.
    For this problem the two largest eigenvalues are 0.8202 and 0.8195, so plain power
    iteration only settles to about 1e-3 in a few hundred cycles."""
    n = 15
    s = O.q1_rotated_stencil(0.01, math.pi / 6)
    mg = O.Multigrid(O.const_field(n, s), coarsest_n=3)
    rho = max(abs(np.linalg.eigvals(D.vcycle_matrix(D.const_matrix(s, n), [15, 7, 3]))))
    zero = np.zeros((n, n))
    op = spla.LinearOperator((n * n, n * n), matvec=lambda v: mg.vcycle(zero, v.reshape(n, n)).ravel(),
                             dtype=np.float64)
    top = spla.eigs(op, k=4, which="LM", return_eigenvectors=False, tol=1e-12)
    assert abs(max(abs(top)) - rho) < 1e-9
    x = np.random.default_rng(0).standard_normal((n, n))
    ratios = []
    for _ in range(400):
        y = mg.vcycle(zero, x)
        ratios.append(np.linalg.norm(y) / np.linalg.norm(x))
        x = y / np.linalg.norm(y)
    factor = math.exp(np.mean(np.log(ratios[100:])))
    assert abs(factor - rho) < 1e-3 * rho


def test_solve_reaches_tolerance_and_direct_solution():
    """63 x 63 rotated problem (eps = 0.01, theta = pi/6): the solve history ends below
    1e-8 and x agrees with a sparse direct solve."""
    n = 63
    s = O.q1_rotated_stencil(0.01, math.pi / 6).astype(np.float32).astype(np.float64)
    st = O.const_field(n, s)
    mg = O.Multigrid(st)
    assert mg.levels == 5
    b = np.random.default_rng(0).uniform(-1, 1, (n, n)).astype(np.float32).astype(np.float64)
    x, hist = mg.solve(b, rtol=1e-8, max_cycles=1000)
    assert hist[0] == 1.0 and hist[-1] < 1e-8 and hist[-2] >= 1e-8
    xs = spla.spsolve(sp.csr_matrix(D.const_matrix(s, n)), b.ravel())
    assert np.linalg.norm(x.ravel() - xs) / np.linalg.norm(xs) < 1e-6
    # the recorded history is the true relative residual of the iterate
    assert abs(np.linalg.norm(b - O.apply(st, x)) / np.linalg.norm(b) - hist[-1]) < 1e-15


def test_linearity_and_scale_invariance():
    n = 31
    rng = np.random.default_rng(4)
    s = O.q1_rotated_stencil(0.1, 0.7)
    st = O.const_field(n, s)
    mg = O.Multigrid(st)
    b, x = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    # V(x, b) = x + V(0, b - A x)
    v1 = mg.vcycle(b, x)
    v2 = x + mg.vcycle(b - O.apply(st, x), np.zeros((n, n)))
    np.testing.assert_allclose(v1, v2, atol=1e-10)
    # A -> c A leaves the residual history unchanged
    _, h1 = mg.solve(b, max_cycles=20, rtol=0)
    _, h2 = O.Multigrid(O.const_field(n, 7.5 * s)).solve(b, max_cycles=20, rtol=0)
    np.testing.assert_allclose(h1, h2, rtol=1e-9)
    # theta -> theta + pi is the same operator
    np.testing.assert_allclose(O.q1_rotated_stencil(0.1, 0.7 + math.pi), s, atol=1e-14)


def test_coarsest_cholesky_is_exact():
    rng = np.random.default_rng(9)
    for m in (9, 49):
        M = rng.standard_normal((m, m))
        A = M @ M.T + m * np.eye(m)
        L = A.copy()
        assert O.lib().or_cholesky(m, O.oracle._p(L)) == 0
        b = rng.standard_normal(m)
        x = b.copy()
        O.lib().or_cholesky_solve(m, O.oracle._p(L), O.oracle._p(x))
        assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-14


def test_poisson_textbook_convergence():
    """Q1 Poisson with V(1,1) weighted Jacobi converges at about 0.25 per cycle,
    independently of the grid size."""
    for n in (31, 127):
        mg = O.Multigrid(O.const_field(n, O.q1_rotated_stencil(1.0, 0.0)))
        b = np.random.default_rng(1).uniform(-1, 1, (n, n))
        _, h = mg.solve(b, rtol=1e-8, max_cycles=100)
        assert len(h) - 1 <= 14
        assert 0.15 < h[-1] / h[-2] < 0.3
