"""Pins of the oracle's FGMRES (Sec. 6.4), CPU only."""
import math

import numpy as np
import pytest

import oracle as O
from tests import dense_ref as D

scipy_sla = pytest.importorskip("scipy.sparse.linalg")


def _problem(n, eps, theta, seed):
    st = O.const_field(n, O.q1_rotated_stencil(eps, theta))
    b = np.random.default_rng(seed).uniform(-1, 1, (n, n))
    return st, b


def test_identity_preconditioner_is_textbook_gmres():
    """With M = I, flexible GMRES is GMRES: the residual norms of its first restart cycle
    equal those of scipy's GMRES (a library routine) iteration by iteration."""
    n = 15
    st, b = _problem(n, 0.1, 0.5, 1)
    A = D.field_matrix(st)
    _, hist, its = O.fgmres(lambda v: O.apply(st, v), lambda v: v, b, restart=40, rtol=1e-10, max_iters=40)
    ref = []
    scipy_sla.gmres(A, b.ravel(), restart=40, maxiter=1, rtol=1e-10, atol=0.0,
                    callback=lambda rn: ref.append(rn), callback_type="pr_norm")
    k = min(len(ref), its)
    assert k >= 20
    np.testing.assert_allclose(hist[1:k + 1], np.array(ref[:k]), rtol=1e-8)


def test_exact_preconditioner_converges_in_one_iteration():
    n = 15
    st, b = _problem(n, 0.01, math.pi / 6, 2)
    A = D.field_matrix(st)
    x, hist, its = O.fgmres(lambda v: O.apply(st, v), lambda v: np.linalg.solve(A, v.ravel()).reshape(v.shape), b,
                            rtol=1e-10)
    assert its == 1
    assert np.linalg.norm(b.ravel() - A @ x.ravel()) < 1e-12 * np.linalg.norm(b)


def test_multigrid_preconditioned_fgmres_reaches_tolerance_with_true_residual():
    """MG-preconditioned FGMRES (one V-cycle per step): the reported residual is the true one
    at exit, the history is non-increasing (minimal residual over a growing space within a
    restart cycle), and it needs fewer steps than the V-cycle alone to 1e-6."""
    n = 63
    st, b = _problem(n, 0.01, math.pi / 12, 3)
    mg = O.Multigrid(st)
    x, hist, its = O.fgmres(lambda v: O.apply(st, v), lambda v: mg.vcycle(v, np.zeros_like(v)), b, restart=30,
                            rtol=1e-6)
    true = np.linalg.norm(b - O.apply(st, x)) / np.linalg.norm(b)
    assert true < 1e-6 and abs(true - hist[-1]) <= 1e-6 * 1e-3 + 1e-3 * true
    assert np.all(np.diff(hist) <= 1e-12)
    _, mg_hist = mg.solve(b, rtol=1e-6, max_cycles=2000)
    assert its < len(mg_hist) - 1
