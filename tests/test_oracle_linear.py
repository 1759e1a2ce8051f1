"""Pins of the shared-kernel linear smoother oracle (Sec. 6, eq. full-coarsening-smoother).

Each check reaches the oracle from outside it: a library correlation, the adjoint identity,
the C oracle's Jacobi multigrid and loss (an independent implementation that the linear
smoother reduces to exactly), and central finite differences of the loss.
"""
import math

import numpy as np
import pytest
from scipy.signal import correlate2d, convolve2d

import oracle as O
from oracle import linear as OL


def _rng(seed):
    return np.random.default_rng(seed)


def test_one_layer_is_a_zero_padded_correlation():
    rng = _rng(0)
    for n in (1, 2, 5, 9):
        phi = rng.standard_normal(9)
        v = rng.standard_normal((n, n))
        k = phi.reshape(3, 3)
        ref = correlate2d(v, k, mode="same", boundary="fill", fillvalue=0.0)
        assert np.allclose(OL.conv(phi, v), ref, rtol=0, atol=1e-13)
        # the transpose is the convolution with the same kernel (the mirrored correlation)
        ref_t = convolve2d(v, k, mode="same", boundary="fill", fillvalue=0.0)
        assert np.allclose(OL.conv_T(phi, v), ref_t, rtol=0, atol=1e-13)


def test_chain_is_five_layers_plus_a_parallel_one():
    rng = _rng(1)
    n = 11
    phi = rng.standard_normal((6, 9))
    v = rng.standard_normal((n, n))
    ref = v
    for k in range(5):
        ref = correlate2d(ref, phi[k].reshape(3, 3), mode="same", boundary="fill")
    ref = ref + correlate2d(v, phi[5].reshape(3, 3), mode="same", boundary="fill")
    assert np.allclose(OL.apply_H(phi, v), ref, rtol=0, atol=1e-12)


def test_transpose_is_the_adjoint():
    rng = _rng(2)
    n = 9
    phi = rng.standard_normal((6, 9))
    u, w = rng.standard_normal((2, n, n))
    lhs = np.sum(OL.apply_H(phi, u) * w)
    assert math.isclose(lhs, np.sum(u * OL.apply_HT(phi, w)), rel_tol=1e-12)
    # H^T as a chain of the same form (reversed, mirrored kernels)
    assert np.allclose(OL.apply_H(OL.transpose_params(phi), w), OL.apply_HT(phi, w), rtol=0, atol=1e-11)


def test_jacobi_point_reduces_to_weighted_jacobi():
    rng = _rng(3)
    d = 2.7
    phi = OL.jacobi_params(d, 2.0 / 3.0)
    v = rng.standard_normal((7, 7))
    assert np.allclose(OL.apply_H(phi, v), (2.0 / 3.0) / d * v, rtol=0, atol=1e-15)


def _jacobi_levels(mg):
    return [OL.jacobi_params(mg.st[l][4, mg.n(l) // 2, mg.n(l) // 2]) for l in range(mg.L)]


def test_vcycle_history_equals_c_oracle_jacobi_multigrid():
    # C1's problem: 63^2 rotated Q1, eps = 0.01, theta = pi/6, Jacobi omega = 2/3
    n = 63
    st = O.const_field(n, O.q1_rotated_stencil(0.01, math.pi / 6))
    b = _rng(4).uniform(-1, 1, (n, n))
    mgl = OL.LinearMultigrid(st, [np.zeros((6, 9))])
    mgl = OL.LinearMultigrid(st, _jacobi_levels(mgl))
    _, h_lin = mgl.solve(b, rtol=1e-8, max_cycles=60)
    _, h_c = O.Multigrid(st).solve(b, rtol=1e-8, max_cycles=60)
    assert len(h_lin) == len(h_c)
    assert np.max(np.abs(h_lin - h_c) / h_c) < 1e-10


def test_twogrid_loss_at_the_jacobi_point_equals_c_oracle():
    n = 15
    st = O.const_field(n, O.q1_rotated_stencil(0.05, 0.7))
    z = _rng(5).standard_normal((3, n, n))
    d = st[4, n // 2, n // 2]
    phi = OL.jacobi_params(d)
    loss, dphi = OL.loss_and_grad(st, phi, z)
    W = O.jacobi_kernels(st)
    loss_c, dW = O.twogrid_loss(st, W, z, want_grad=True)
    assert math.isclose(loss, loss_c, rel_tol=1e-12)
    # phi_6 acts as one per-point kernel shared by every point: its gradient is the sum of
    # the per-point gradient over the grid
    assert np.allclose(dphi[5], dW.reshape(9, -1).sum(axis=1), rtol=1e-10, atol=1e-14)
    # two cycles: the k-cycle objective of the C oracle
    loss2 = OL.loss_and_grad(st, phi, z, cycles=2, want_grad=False)
    assert math.isclose(loss2, O.twogrid_loss(st, W, z, cycles=2), rel_tol=1e-12)


def _fd_check(fun, phi, rel=1e-6, h=1e-6):
    _, g = fun(phi)
    fd = np.zeros_like(phi)
    for idx in np.ndindex(*phi.shape):
        p = phi.copy()
        p[idx] += h
        lp = fun(p)[0]
        p[idx] -= 2 * h
        lm = fun(p)[0]
        fd[idx] = (lp - lm) / (2 * h)
    scale = np.max(np.abs(fd))
    assert np.max(np.abs(g - fd)) <= rel * scale + 1e-12, np.max(np.abs(g - fd)) / scale


@pytest.mark.parametrize("cycles", [1, 2])
def test_gradient_matches_central_differences(cycles):
    n = 7
    st = O.const_field(n, O.q1_rotated_stencil(0.1, 0.4))
    rng = _rng(6)
    z = rng.standard_normal((2, n, n))
    phi = OL.jacobi_params(st[4, 3, 3]) + 0.1 * rng.standard_normal((6, 9))
    _fd_check(lambda p: OL.loss_and_grad(st, p, z, cycles=cycles), phi)


def test_vcycle_with_transposed_smoothers_is_the_adjoint_cycle():
    rng = _rng(7)
    n = 15
    st = O.const_field(n, O.q1_rotated_stencil(0.02, 1.1))
    phis = [OL.jacobi_params(3.0) + 0.1 * rng.standard_normal((6, 9)) for _ in range(3)]
    M = OL.coarse_vcycle(st, phis)
    MT = OL.coarse_vcycle(st, phis, transpose=True)
    r, s = rng.standard_normal((2, n, n))
    assert math.isclose(np.sum(M(r) * s), np.sum(r * MT(s)), rel_tol=1e-11)


def test_coarse_vcycle_loss_gradient_matches_central_differences():
    # Algorithm 2 on a 15^2 level: coarse solve = one V-cycle of the trained 7^2 hierarchy
    rng = _rng(8)
    n = 15
    st = O.const_field(n, O.q1_rotated_stencil(0.05, 2.0))
    st_c = O.rap(st)
    lower = [OL.jacobi_params(st_c[4, 3, 3]) + 0.05 * rng.standard_normal((6, 9))]
    coarse = OL.coarse_vcycle(st_c, lower)
    coarse_t = OL.coarse_vcycle(st_c, lower, transpose=True)
    z = rng.standard_normal((1, n, n))
    phi = OL.jacobi_params(st[4, 7, 7]) + 0.05 * rng.standard_normal((6, 9))
    _fd_check(lambda p: OL.loss_and_grad(st, p, z, cycles=1, coarse=coarse, coarse_t=coarse_t), phi)


def test_multistep_smoothing_at_the_jacobi_point_equals_c_oracle():
    """nu1, nu2 > 1 (Algorithm 1's smoothing steps): the linear oracle at the Jacobi point
    against the C oracle's Jacobi multigrid with the same steps."""
    n = 31
    st = O.const_field(n, O.q1_rotated_stencil(0.05, 0.9))
    b = _rng(9).uniform(-1, 1, (n, n))
    base = OL.LinearMultigrid(st, [np.zeros((6, 9))])
    for nu1, nu2 in ((2, 2), (3, 1), (6, 6)):
        mgl = OL.LinearMultigrid(st, _jacobi_levels(base), nu1=nu1, nu2=nu2)
        _, hl = mgl.solve(b, rtol=0.0, max_cycles=8)
        _, hc = O.Multigrid(st, nu1=nu1, nu2=nu2).solve(b, rtol=0.0, max_cycles=8)
        assert np.max(np.abs(hl - hc) / hc) < 1e-10
