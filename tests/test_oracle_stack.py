"""Pins of the k = 3 stack oracle (Sec. 4, Sec. 4.2: three output kernels per point).

The stack reduces to the k = 1 network when the last layer's rows of kernels 2 and 3 are
zero; there the oracle must agree with the independent C oracle (network, loss, gradient).
Its operators are checked against the C oracle's, the stack's transpose by the adjoint
identity, kernels 2 and 3 against the C oracle's network on their rows of the last layer,
the loss at a general point against dense error-propagation matrices, and the remaining
gradient by central differences.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import stack as OS
from tests import dense_ref as D


def _rng(seed):
    return np.random.default_rng(seed)


def _params(seed, scale=0.3, zero_rest=False):
    p = _rng(seed).standard_normal(OS.NPARAMS) * scale
    if zero_rest:
        p[-18 * 27:] = 0.0  # rows of kernels 2 and 3 in the last layer
    return p


def test_parameter_count():
    assert OS.NPARAMS == 1017 + 27 * 27 == 1746
    assert OS.k1_params(np.zeros(OS.NPARAMS)).size == O.hypernet_nparams()


def test_stack_reduces_to_the_k1_network_of_the_c_oracle():
    n = 11
    st = O.varcoef5_field(n, np.exp(_rng(1).standard_normal((n + 1, n + 1))))
    p = _params(2, zero_rest=True)
    K = OS.kernels(st, torch.from_numpy(p)).numpy()
    W = O.hypernet_forward(st, OS.k1_params(p))
    assert np.allclose(K[0], W, rtol=1e-12, atol=1e-14)
    delta = np.zeros((9, n, n))
    delta[4] = 1.0
    assert np.array_equal(K[1], delta) and np.array_equal(K[2], delta)


def test_operators_match_the_c_oracle():
    rng = _rng(3)
    n = 15
    st = O.const_field(n, O.q1_rotated_stencil(0.05, 0.4))
    v = rng.standard_normal((n, n))
    W = rng.standard_normal((9, n, n))
    tv = torch.from_numpy(v)
    assert np.allclose(OS.apply_A(st, tv).numpy(), O.apply(st, v), rtol=0, atol=1e-12)
    assert np.allclose(OS.apply_kernel(torch.from_numpy(W), tv).numpy(), O.apply_H(W, v), rtol=0, atol=1e-12)
    assert np.allclose(OS.apply_kernel_T(torch.from_numpy(W), tv).numpy(), O.apply_HT(W, v), rtol=0, atol=1e-12)
    assert np.allclose(OS.restrict(tv).numpy(), O.restrict(v), rtol=0, atol=1e-12)
    ec = rng.standard_normal(((n - 1) // 2, (n - 1) // 2))
    assert np.allclose(OS.prolong(torch.from_numpy(ec), n).numpy(), O.prolong(ec, n), rtol=0, atol=1e-12)


def test_stack_is_three_chained_kernels_and_its_transpose_the_adjoint():
    rng = _rng(4)
    n = 9
    Ks = torch.from_numpy(rng.standard_normal((3, 9, n, n)))
    u, w = (torch.from_numpy(a) for a in rng.standard_normal((2, n, n)))
    ref = O.apply_H(Ks[2].numpy(), O.apply_H(Ks[1].numpy(), O.apply_H(Ks[0].numpy(), u.numpy())))
    assert np.allclose(OS.apply_H(Ks, u).numpy(), ref, rtol=0, atol=1e-11)
    lhs = float((OS.apply_H(Ks, u) * w).sum())
    assert math.isclose(lhs, float((u * OS.apply_HT(Ks, w)).sum()), rel_tol=1e-12)


def test_loss_and_gradient_at_the_k1_point_equal_the_c_oracle():
    n = 15
    st = O.const_field(n, O.q1_rotated_stencil(0.05, 0.7))
    z = _rng(5).standard_normal((2, n, n))
    p = _params(6, scale=0.05, zero_rest=True)
    L, g = OS.loss_and_grad(st, O.rap(st), p, z)
    Lc, gc = O.cnn_loss_and_grad(st, OS.k1_params(p), z)
    assert math.isclose(L, Lc, rel_tol=1e-11)
    assert np.allclose(OS.k1_params(g), gc, rtol=1e-8, atol=1e-12 * np.abs(gc).max())


def test_gradient_matches_central_differences():
    n = 7
    st = O.varcoef5_field(n, np.exp(0.5 * _rng(7).standard_normal((n + 1, n + 1))))
    stc = O.rap(st)
    z = _rng(8).standard_normal((2, n, n))
    p = _params(9, scale=0.05)
    _, g = OS.loss_and_grad(st, stc, p, z, cycles=2)
    idx = _rng(10).choice(OS.NPARAMS, 40, replace=False)
    idx = np.concatenate([idx, np.arange(OS.NPARAMS - 30, OS.NPARAMS)])  # include kernels 2, 3
    h = 1e-6
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        lp = float(OS.loss(st, stc, torch.from_numpy(pp), z, cycles=2))
        lm = float(OS.loss(st, stc, torch.from_numpy(pm), z, cycles=2))
        fd = (lp - lm) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * np.abs(g).max() + 1e-10, (k, g[k], fd)


def test_stack_vcycle_reduces_to_the_c_oracle_cnn_multigrid():
    """Algorithm 1 with the stack smoother on every level: at the k = 1 point its history is
    the C oracle's CNN-smoothed multigrid's."""
    n = 31
    st = O.const_field(n, O.q1_rotated_stencil(0.05, 1.2))
    b = _rng(11).uniform(-1, 1, (n, n))
    p = _params(12, scale=0.05, zero_rest=True)
    sm = OS.StackMultigrid(st, p)
    _, hs = sm.solve(b, rtol=0.0, max_cycles=10)
    mg = O.Multigrid(st)
    mg.set_cnn(OS.k1_params(p))
    _, hc = mg.solve(b, rtol=0.0, max_cycles=10)
    assert np.max(np.abs(hs - hc) / hc) < 1e-10
    # one cycle from zero, the FGMRES preconditioner, is the C oracle's as well
    np.testing.assert_allclose(sm.vcycle(b, np.zeros_like(b)), mg.vcycle(b, np.zeros_like(b)), rtol=0, atol=1e-12)
    # with the other two kernels in play the smoother differs, and the cycle still runs
    _, h3 = OS.StackMultigrid(st, _params(12, scale=0.05)).solve(b, rtol=0.0, max_cycles=3)
    assert np.all(np.isfinite(h3)) and abs(h3[1] - hc[1]) > 1e-6


def test_kernels_two_and_three_are_the_k1_network_on_their_rows_of_the_last_layer():
    """out_k (k = 2, 3) is the k = 1 network of the C oracle whose last layer is the stack's
    rows 9(k-1) .. 9k-1: recovered from W = (omega delta + out)/D as out = D W - omega delta."""
    n, omega = 11, 0.6
    st = O.varcoef5_field(n, np.exp(_rng(20).standard_normal((n + 1, n + 1))))
    p = _params(21)
    K = OS.kernels(st, torch.from_numpy(p), omega).numpy()
    conv = p[:1017]
    wf = p[1017:].reshape(27, 27)
    delta = np.zeros((9, 1, 1))
    delta[4] = 1.0
    for k in (1, 2):
        W = O.hypernet_forward(st, np.concatenate([conv, wf[9 * k:9 * k + 9].ravel()]), omega)
        out = W * st[4] - omega * delta
        np.testing.assert_allclose(K[k], delta + out, rtol=1e-12, atol=1e-12 * np.abs(out).max())


@pytest.mark.parametrize("cycles", [1, 2])
def test_loss_is_the_dense_error_propagation_of_the_stack(cycles):
    """The loss at a general point (all three kernels active) against dense matrices:
    H = K3 K2 K1 from per-point kernel matrices, S = I - H A, C = I - P Ac^-1 P^T A."""
    n = 7
    st = O.varcoef5_field(n, np.exp(0.5 * _rng(22).standard_normal((n + 1, n + 1))))
    stc = O.rap(st)
    p = _params(23, scale=0.1)
    z = _rng(24).standard_normal((3, n, n))
    K = OS.kernels(st, torch.from_numpy(p)).numpy()
    A = D.field_matrix(st)
    H = D.kernels_matrix(K[2]) @ D.kernels_matrix(K[1]) @ D.kernels_matrix(K[0])
    P = D.prolongation(n)
    I = np.eye(n * n)
    S = I - H @ A
    C = I - P @ np.linalg.solve(P.T @ A @ P, P.T @ A)
    E = np.linalg.matrix_power(S @ C @ S, cycles)
    ref = np.mean([np.sum((E @ zj.ravel()) ** 2) for zj in z]) / (n * n)
    L = float(OS.loss(st, stc, torch.from_numpy(p), z, cycles=cycles))
    assert math.isclose(L, ref, rel_tol=1e-11), (L, ref)


def test_algorithm2_objective_at_the_k1_point_equals_the_c_oracle():
    """Algorithm 2's objective with the stack (coarse solve = one V-cycle of stack smoothers
    on the coarse hierarchy, its adjoint by autograd) at the k = 1 point, where every stack
    is the k = 1 network's kernel: loss and gradient equal the C oracle's vcycle objective,
    whose adjoint is the explicitly transposed-kernel cycle."""
    n = 31
    st = O.const_field(n, O.q1_rotated_stencil(0.1, 1.1))
    st_c = O.rap(st)
    z = _rng(11).standard_normal((2, n, n))
    p = _params(12, scale=0.05, zero_rest=True)
    sets = [_params(13 + j, scale=0.05, zero_rest=True) for j in range(2)]
    L, g = OS.loss_and_grad(st, st_c, p, z, coarse=OS.coarse_vcycle(st_c, sets))
    mgc = O.Multigrid(st_c)
    ker = [O.hypernet_forward(mgc.field(j), OS.k1_params(sets[min(j, 1)])) for j in range(mgc.levels - 1)]
    Lc, gc = O.vcycle_cnn_loss_and_grad(st, OS.k1_params(p), O.coarse_vcycle(st_c, ker),
                                        O.coarse_vcycle(st_c, ker, transpose=True), z)
    assert math.isclose(L, Lc, rel_tol=1e-10)
    assert np.allclose(OS.k1_params(g), gc, rtol=1e-7, atol=1e-11 * np.abs(gc).max())


def test_coarse_vcycle_is_the_stack_multigrid_cycle_and_exact_on_the_coarsest():
    """The torch coarse V-cycle against the numpy StackMultigrid cycle from zero (general
    stack), and, on a coarse grid that is the coarsest (side 3), the exact solve: there
    Algorithm 2's objective is the two-grid one."""
    nc = 15
    st_c = O.varcoef5_field(nc, np.exp(_rng(14).standard_normal((nc + 1, nc + 1))))
    p = _params(15, scale=0.1)
    r = _rng(16).standard_normal((nc, nc))
    got = OS.coarse_vcycle(st_c, [p])(torch.from_numpy(r)).numpy()
    want = OS.StackMultigrid(st_c, p).vcycle(r, np.zeros_like(r))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
    n = 7
    st = O.const_field(n, O.q1_rotated_stencil(0.3, 0.4))
    z = _rng(17).standard_normal((2, n, n))
    q = _params(18, scale=0.1)
    L1 = OS.loss(st, O.rap(st), torch.from_numpy(q), z, coarse=OS.coarse_vcycle(O.rap(st), [q])).item()
    L0 = OS.loss(st, O.rap(st), torch.from_numpy(q), z).item()
    assert math.isclose(L1, L0, rel_tol=1e-12)


def test_algorithm2_gradient_matches_central_differences():
    n = 15
    st = O.varcoef5_field(n, np.exp(0.5 * _rng(19).standard_normal((n + 1, n + 1))))
    st_c = O.rap(st)
    z = _rng(20).standard_normal((2, n, n))
    p = _params(21, scale=0.1)
    cv = OS.coarse_vcycle(st_c, [_params(22, scale=0.1)])
    _, g = OS.loss_and_grad(st, st_c, p, z, coarse=cv)
    d = _rng(23).standard_normal(p.size)
    h = 1e-6
    lp = OS.loss(st, st_c, torch.from_numpy(p + h * d), z, coarse=cv).item()
    lm = OS.loss(st, st_c, torch.from_numpy(p - h * d), z, coarse=cv).item()
    assert math.isclose((lp - lm) / (2 * h), g @ d, rel_tol=1e-6)
