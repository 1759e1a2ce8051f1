"""Pins of the oracle's discretisations, operators and transfers (no GPU).

Each test checks the oracle against something fixed outside it: numbers printed in
the paper, closed forms, a different matrix formulation, or known eigenpairs.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from tests import dense_ref as D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_spectral_radius.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                xi, th, rj, rg = (float(v) for v in line.split())
                rows.append((xi, th * math.pi, rj, rg))
    return rows


@pytest.mark.parametrize("xi,theta,rho_j,rho_gs", _table1())
def test_table1_jacobi_and_gauss_seidel(xi, theta, rho_j, rho_gs):
    """Sec. 6.1 Table 1: rho(I - omega D^-1 A) and rho(I - (D-L)^-1 A) on a 16 x 16 grid,
    using the oracle's FD stencil, its Jacobi kernels and its Gauss-Seidel sweep."""
    n = 16
    st = O.const_field(n, O.fd_rotated_stencil(xi, theta))
    # iteration matrices built column by column from the oracle's own smoother sweeps
    Wj = O.jacobi_kernels(st, 2.0 / 3.0)
    GJ = np.zeros((n * n, n * n))
    GG = np.zeros((n * n, n * n))
    zero = np.zeros((n, n))
    for c in range(n * n):
        e = np.zeros(n * n)
        e[c] = 1.0
        GJ[:, c] = O.smooth(st, Wj, zero, e.reshape(n, n)).ravel()
        GG[:, c] = O.gauss_seidel(st, zero, e.reshape(n, n)).ravel()
    assert abs(max(abs(np.linalg.eigvals(GJ))) - rho_j) < 5.1e-5
    assert abs(max(abs(np.linalg.eigvals(GG))) - rho_gs) < 5.1e-5


def test_jacobi_closed_form_theta0():
    """theta = 0: rho_J = 1 - omega (1 - cos(pi h)), h = 1/17, for every xi (Table 1 row)."""
    n = 16
    for xi in (1.0, 100.0, 400.0):
        A = D.const_matrix(O.fd_rotated_stencil(xi, 0.0), n)
        G = np.eye(n * n) - (2.0 / 3.0) * np.diag(1.0 / np.diag(A)) @ A
        rho = max(abs(np.linalg.eigvals(G)))
        assert abs(rho - (1.0 - (2.0 / 3.0) * (1.0 - math.cos(math.pi / 17)))) < 1e-12


@pytest.mark.parametrize("eps,theta", [(1.0, 0.0), (0.01, math.pi / 6), (1e-3, 2.0), (0.3, 5 * math.pi / 12)])
def test_q1_rotated_closed_form(eps, theta):
    """The oracle assembles Q1 element matrices by quadrature; the interior stencil must
    equal the closed form of the Q1 rotated-anisotropic stencil (derived by hand)."""
    a = math.cos(theta) ** 2 + eps * math.sin(theta) ** 2
    c = math.sin(theta) ** 2 + eps * math.cos(theta) ** 2
    b = math.cos(theta) * math.sin(theta) * (1 - eps)
    s = O.q1_rotated_stencil(eps, theta)  # rows: south, centre, north
    want = np.array([
        [-(a + c) / 6 - b / 2, (a - 2 * c) / 3, -(a + c) / 6 + b / 2],
        [(c - 2 * a) / 3, 4 * (a + c) / 3, (c - 2 * a) / 3],
        [-(a + c) / 6 + b / 2, (a - 2 * c) / 3, -(a + c) / 6 - b / 2],
    ])
    np.testing.assert_allclose(s, want, atol=1e-15)
    assert abs(s.sum()) < 1e-14  # constants are in the kernel of the continuous operator


def test_q1_laplacian_and_paper_nine_point():
    """Isotropic cellwise coefficient: the printed nine-point formula of Sec. 4 must equal
    the oracle's Q1 assembly; for g = 1 it is the Q1 Laplacian [-1 -1 -1; -1 8 -1; -1 -1 -1]/3."""
    np.testing.assert_allclose(O.q1_rotated_stencil(1.0, 0.3) * 3, [[-1, -1, -1], [-1, 8, -1], [-1, -1, -1]], atol=1e-14)
    n = 9
    g = np.random.default_rng(5).uniform(0.5, 2.0, (n + 1, n + 1))
    fe = O.fe_q1_field(n, g, np.zeros_like(g), g)
    np.testing.assert_allclose(O.paper9_field(n, g), fe, atol=1e-14)


def test_varcoef5_constant_is_five_point_laplacian():
    n = 7
    st = O.varcoef5_field(n, np.ones((n + 1, n + 1)))
    np.testing.assert_allclose(D.field_matrix(st), D.const_matrix([0, -1, 0, -1, 4, -1, 0, -1, 0], n), atol=0)


def test_varcoef5_second_order_consistency():
    """(A u)/h^2 -> -div(a grad u) at rate h^2 for smooth a, u (a sampled at cell centres)."""
    errs = []
    for n in (15, 31, 63):
        h = 1.0 / (n + 1)
        xc = (np.arange(n + 1) + 0.5) * h
        Yc, Xc = np.meshgrid(xc, xc, indexing="ij")
        a = 1.0 + Xc + Yc ** 2
        st = O.varcoef5_field(n, a)
        x = (np.arange(n) + 1) * h
        Y, X = np.meshgrid(x, x, indexing="ij")
        u = np.sin(math.pi * X) * np.sin(math.pi * Y)
        # -div(a grad u) with a = 1 + x + y^2, a_x = 1, a_y = 2y
        ux = math.pi * np.cos(math.pi * X) * np.sin(math.pi * Y)
        uy = math.pi * np.sin(math.pi * X) * np.cos(math.pi * Y)
        lap = -2 * math.pi ** 2 * u
        f = -((1.0 + X + Y ** 2) * lap + 1.0 * ux + 2 * Y * uy)
        errs.append(np.abs(O.apply(st, u) / h ** 2 - f).max())
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_apply_matches_shift_matrix_form():
    rng = np.random.default_rng(1)
    for n in (5, 8):
        st = O.const_field(n, rng.standard_normal(9))
        st *= rng.uniform(0.5, 1.5, st.shape)  # make it genuinely per-point
        x = rng.standard_normal((n, n))
        np.testing.assert_allclose(O.apply(st, x).ravel(), D.field_matrix(st) @ x.ravel(), atol=1e-13)
        np.testing.assert_allclose(O.dense_matrix(st), D.field_matrix(st), atol=0)


def test_transfers_are_kronecker_interpolation():
    rng = np.random.default_rng(2)
    for n in (7, 15):
        nc = (n - 1) // 2
        P = D.prolongation(n)
        ec = rng.standard_normal((nc, nc))
        r = rng.standard_normal((n, n))
        np.testing.assert_allclose(O.prolong(ec, n).ravel(), P @ ec.ravel(), atol=1e-14)
        np.testing.assert_allclose(O.restrict(r).ravel(), P.T @ r.ravel(), atol=1e-14)
        # <P v, w> = <v, P^T w>
        assert abs(np.vdot(O.prolong(ec, n), r) - np.vdot(ec, O.restrict(r))) < 1e-12


def test_rap_matches_dense_galerkin():
    rng = np.random.default_rng(3)
    n = 15
    fields = [
        O.varcoef5_field(n, np.exp(rng.standard_normal((n + 1, n + 1)))),
        O.paper9_field(n, rng.uniform(0.1, 3, (n + 1, n + 1))),
        O.const_field(n, O.q1_rotated_stencil(0.05, 1.1)),
    ]
    P = D.prolongation(n)
    for st in fields:
        stc = O.rap(st)
        np.testing.assert_allclose(D.field_matrix(stc), P.T @ D.field_matrix(st) @ P, atol=1e-12)


@pytest.mark.parametrize("eps,theta", [(1.0, 0.0), (0.01, math.pi / 6), (1e-3, 2.5)])
def test_q1_galerkin_invariance(eps, theta):
    """Nested Q1 spaces: P^T A P of the constant Q1 stencil is the same stencil one level down."""
    n = 31
    s = O.q1_rotated_stencil(eps, theta)
    stc = O.rap(O.const_field(n, s))
    np.testing.assert_allclose(stc, O.const_field(15, s), atol=1e-14)


def test_jacobi_eigenpairs_five_point():
    """Sine modes are eigenvectors of I - omega D^-1 A for the 5-point Laplacian with
    eigenvalue 1 - omega (1 - (cos k pi h + cos l pi h)/2); the LFA smoothing factor 2/3
    for omega = 2/3 is the largest such value over the high-frequency half."""
    n, omega = 15, 2.0 / 3.0
    h = 1.0 / (n + 1)
    st = O.varcoef5_field(n, np.ones((n + 1, n + 1)))
    W = O.jacobi_kernels(st, omega)
    i = np.arange(1, n + 1) * h
    mu = 0.0
    for k in (1, 3, 8, 12, 15):
        for l in (1, 5, 9, 15):
            v = np.outer(np.sin(k * math.pi * i), np.sin(l * math.pi * i))
            lam = 1 - omega * (1 - (math.cos(k * math.pi * h) + math.cos(l * math.pi * h)) / 2)
            np.testing.assert_allclose(O.smooth(st, W, np.zeros((n, n)), v), lam * v, atol=1e-13)
            if max(k, l) > (n + 1) // 2:
                mu = max(mu, abs(lam))
    # continuous LFA limit: max over high frequencies of |1 - omega (1 - (cos a + cos b)/2)| = 2/3
    t = np.linspace(-math.pi, math.pi, 401)
    A_, B_ = np.meshgrid(t, t)
    hi = np.maximum(abs(A_), abs(B_)) >= math.pi / 2
    lfa = np.abs(1 - omega * (1 - (np.cos(A_) + np.cos(B_)) / 2))[hi].max()
    assert abs(lfa - 2.0 / 3.0) < 1e-12 and mu <= lfa + 1e-12


@pytest.mark.parametrize("eps,theta", [(0.01, math.pi / 6), (0.2, 1.1), (0.05, 2.7)])
def test_orientation_mirror_and_transpose_symmetries(eps, theta):
    """The orientation convention (row index = y, column = x) is immaterial: mirroring the
    grid in x is K(theta) -> K(-theta) (the cross term changes sign) and swapping x and y is
    theta -> pi/2 - theta, for the operator and for whole V-cycle solves (same histories,
    mirrored or transposed iterates).  The parametrisation itself is pinned by the closed
    form above."""
    n = 31
    rng = np.random.default_rng(40)
    u = rng.standard_normal((n, n))
    A = O.q1_rotated_stencil(eps, theta)
    A_m = O.q1_rotated_stencil(eps, -theta)
    A_t = O.q1_rotated_stencil(eps, math.pi / 2 - theta)
    Au = O.apply(O.const_field(n, A), u)
    np.testing.assert_allclose(O.apply(O.const_field(n, A_m), u[:, ::-1])[:, ::-1], Au, rtol=0, atol=1e-13)
    np.testing.assert_allclose(O.apply(O.const_field(n, A_t), u.T).T, Au, rtol=0, atol=1e-13)
    b = rng.uniform(-1, 1, (n, n))
    x, h = O.Multigrid(O.const_field(n, A)).solve(b, rtol=0.0, max_cycles=6)
    x_m, h_m = O.Multigrid(O.const_field(n, A_m)).solve(np.ascontiguousarray(b[:, ::-1]), rtol=0.0, max_cycles=6)
    x_t, h_t = O.Multigrid(O.const_field(n, A_t)).solve(np.ascontiguousarray(b.T), rtol=0.0, max_cycles=6)
    np.testing.assert_allclose(h_m, h, rtol=1e-10)
    np.testing.assert_allclose(h_t, h, rtol=1e-10)
    np.testing.assert_allclose(x_m[:, ::-1], x, rtol=0, atol=1e-10 * np.abs(x).max())
    np.testing.assert_allclose(x_t.T, x, rtol=0, atol=1e-10 * np.abs(x).max())
