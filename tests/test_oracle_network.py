"""Pins of the oracle's stencil-to-smoother network and the training loss (no GPU).

The network is checked against torch's float64 conv2d / autograd (library routines);
the loss against dense error-propagation matrices; its gradient against central
finite differences; and its normalisation against the Frobenius identity of Thm. sbound.
"""
import math

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle as O
from tests import dense_ref as D

NP = 7 * 9 * 9 + 5 * 7 * 9 + 3 * 5 * 9 + 9 * 3 * 9


def _split(p):
    p = torch.as_tensor(p)
    sizes = [(7, 9, 3, 3), (5, 7, 3, 3), (3, 5, 3, 3), (9, 3, 3, 3)]
    out, o = [], 0
    for s in sizes:
        k = int(np.prod(s))
        out.append(p[o:o + k].reshape(s))
        o += k
    return out


def _torch_net(st, params, omega=2.0 / 3.0, bf16=False):
    """Reference forward with torch conv2d; rounding via torch's bfloat16 conversion."""
    rnd = (lambda t: t.to(torch.float32).to(torch.bfloat16).to(torch.float64)) if bf16 else (lambda t: t)
    st = torch.as_tensor(st)
    w1, w2, w3, wf = (rnd(w) for w in _split(params))
    x = rnd(st / st[4])[None]
    for w in (w1, w2, w3):
        x = rnd(F.leaky_relu(F.conv2d(x, w, padding=1), 0.01))
    out = F.conv2d(x, wf, padding=1)[0]
    delta = torch.zeros(9, 1, 1, dtype=torch.float64)
    delta[4] = omega
    return (delta + out) / st[4]


def _field(n, seed):
    rng = np.random.default_rng(seed)
    return O.varcoef5_field(n, np.exp(rng.standard_normal((n + 1, n + 1)))) + \
        0.2 * O.paper9_field(n, rng.uniform(0.5, 2.0, (n + 1, n + 1)))


def test_parameter_count():
    # dense 3x3 convolutions 9->7->5->3 plus the 27 -> 9 layer (no biases)
    assert O.hypernet_nparams() == NP == 1260
    # the paper quotes 378 = (7+5+3)*9 + 27*9 (Sec. 6.2): one 3x3 kernel per output channel
    assert (7 + 5 + 3) * 9 + 27 * 9 == 378


def test_zero_last_layer_is_weighted_jacobi():
    n = 11
    st = _field(n, 0)
    p = np.random.default_rng(1).standard_normal(NP)
    p[-243:] = 0.0
    np.testing.assert_array_equal(O.hypernet_forward(st, p, 2.0 / 3.0), O.jacobi_kernels(st, 2.0 / 3.0))


@pytest.mark.parametrize("bf16", [False, True])
def test_forward_matches_torch_conv2d(bf16):
    n = 13
    st = _field(n, 2)
    p = np.random.default_rng(3).standard_normal(NP) * 0.3
    if bf16:  # keep values exactly representable in float32 so both roundings agree
        st = st.astype(np.float32).astype(np.float64)
        p = p.astype(np.float32).astype(np.float64)
    W = O.hypernet_forward(st, p, 0.7, bf16)
    Wt = _torch_net(st, p, 0.7, bf16).numpy()
    if bf16:
        # intermediate values computed in float64 vs float64: identical rounding except
        # at exact ties, which random data does not produce
        np.testing.assert_allclose(W, Wt, rtol=1e-12, atol=1e-13)
    else:
        np.testing.assert_allclose(W, Wt, rtol=1e-12, atol=1e-14)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(4)
    v = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-6, 6, 2000),
                        [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0]]).astype(np.float32)
    mine = np.array([O.bf16(float(x)) for x in v])
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mine, ref)


def test_backward_matches_autograd():
    n = 9
    st = _field(n, 5)
    p = np.random.default_rng(6).standard_normal(NP) * 0.3
    dW = np.random.default_rng(7).standard_normal((9, n, n))
    g = O.hypernet_backward(st, p, dW, 0.7)
    pt = torch.tensor(p, requires_grad=True)
    W = _torch_net(st, pt, 0.7)
    (W * torch.as_tensor(dW)).sum().backward()
    np.testing.assert_allclose(g, pt.grad.numpy(), rtol=1e-10, atol=1e-12)


def _dense_E(st, W):
    n = st.shape[1]
    A = D.field_matrix(st)
    H = D.kernels_matrix(W)
    P = D.prolongation(n)
    I = np.eye(n * n)
    S = I - H @ A
    C = I - P @ np.linalg.solve(P.T @ A @ P, P.T @ A)
    return S @ C @ S


def test_twogrid_loss_matches_dense_error_propagation():
    n = 15
    st = O.const_field(n, O.q1_rotated_stencil(0.05, 1.0))
    W = O.jacobi_kernels(st) * (1 + 0.1 * np.random.default_rng(8).standard_normal((9, n, n)))
    z = np.random.default_rng(9).standard_normal((4, n, n))
    E = _dense_E(st, W)
    want = np.mean([np.sum((E @ zi.ravel()) ** 2) / (n * n) for zi in z])
    assert abs(O.twogrid_loss(st, W, z) - want) < 1e-12 * want
    # dLoss/dW through the dense form: dL/dH = sum_z (2/(Z n)) [S C]^T... checked by FD below


def test_loss_gradient_matches_finite_differences():
    """C3 gradient check: FP64 central differences, h = 1e-6, on a 15 x 15 grid."""
    n = 15
    rng = np.random.default_rng(10)
    eps, theta = 10 ** rng.uniform(-3, 0), rng.uniform(0, math.pi)
    st = O.const_field(n, O.q1_rotated_stencil(eps, theta))
    p = rng.standard_normal(NP) * 0.2
    z = rng.standard_normal((3, n, n))
    loss, g = O.cnn_loss_and_grad(st, p, z)
    h = 1e-6
    idx = list(rng.choice(NP, 12, replace=False)) + [NP - 1, NP - 243, 0]
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        lp = O.twogrid_loss(st, O.hypernet_forward(st, pp), z)
        lm = O.twogrid_loss(st, O.hypernet_forward(st, pm), z)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g).max(), 1e-12), (i, fd, g[i])
    # directional derivative along a random direction
    d = rng.standard_normal(NP)
    lp = O.twogrid_loss(st, O.hypernet_forward(st, p + h * d), z)
    lm = O.twogrid_loss(st, O.hypernet_forward(st, p - h * d), z)
    assert abs((lp - lm) / (2 * h) - g @ d) <= 1e-6 * abs(g @ d)


def test_loss_estimates_frobenius_norm():
    """Thm. sbound: E ||X z||^2 = ||X||_F^2 for Gaussian z; the loss is ||E||_F^2 / n."""
    n = 7
    st = O.const_field(n, O.q1_rotated_stencil(0.02, 0.4))
    W = O.jacobi_kernels(st)
    E = _dense_E(st, W)
    fro = np.sum(E ** 2) / (n * n)
    Z = 4000
    z = np.random.default_rng(11).standard_normal((Z, n, n))
    est = O.twogrid_loss(st, W, z)
    # per-sample variance of ||E z||^2 is 2 ||E^T E||_F^2; 5 standard errors
    sd = math.sqrt(2 * np.sum((E.T @ E) ** 2)) / (n * n) / math.sqrt(Z)
    assert abs(est - fro) < 5 * sd


@pytest.mark.parametrize("cycles", [2, 3])
def test_k_cycle_loss_matches_dense_power(cycles):
    """The k-cycle objective against the dense matrix power: (1/Z) sum ||E^k z||^2 / n^2."""
    n = 15
    st = O.const_field(n, O.q1_rotated_stencil(0.05, 1.0))
    W = O.jacobi_kernels(st) * (1 + 0.1 * np.random.default_rng(12).standard_normal((9, n, n)))
    z = np.random.default_rng(13).standard_normal((4, n, n))
    Ek = np.linalg.matrix_power(_dense_E(st, W), cycles)
    want = np.mean([np.sum((Ek @ zi.ravel()) ** 2) / (n * n) for zi in z])
    assert abs(O.twogrid_loss(st, W, z, cycles=cycles) - want) < 1e-12 * want


def test_k_cycle_loss_with_one_cycle_is_the_two_grid_loss():
    n = 15
    st = O.const_field(n, O.q1_rotated_stencil(0.3, 2.0))
    W = O.jacobi_kernels(st) * (1 + 0.1 * np.random.default_rng(14).standard_normal((9, n, n)))
    z = np.random.default_rng(15).standard_normal((3, n, n))
    l1, g1 = O.twogrid_loss(st, W, z, want_grad=True)
    # the k-cycle routine itself, called with k = 1
    from oracle import oracle as OM

    dW = np.zeros((9, n, n))
    lk = OM.lib().or_twogrid_loss_k(n, OM._p(OM._f64(st)), OM._p(OM._f64(W)), 3, OM._p(OM._f64(z)), 1, OM._p(dW))
    assert lk == l1
    np.testing.assert_array_equal(dW, g1)


def test_k_cycle_gradient_matches_finite_differences():
    """dloss/dparams of the 3-cycle objective against FP64 central differences (h = 1e-6)."""
    n = 15
    rng = np.random.default_rng(16)
    st = O.const_field(n, O.q1_rotated_stencil(10 ** rng.uniform(-3, 0), rng.uniform(0, math.pi)))
    p = rng.standard_normal(NP) * 0.2
    z = rng.standard_normal((2, n, n))
    loss, g = O.cnn_loss_and_grad(st, p, z, cycles=3)
    h = 1e-6
    for i in list(rng.choice(NP, 10, replace=False)) + [NP - 1, 0]:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (O.twogrid_loss(st, O.hypernet_forward(st, pp), z, cycles=3)
              - O.twogrid_loss(st, O.hypernet_forward(st, pm), z, cycles=3)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g).max(), 1e-12), (i, fd, g[i])
    d = rng.standard_normal(NP)
    lp = O.twogrid_loss(st, O.hypernet_forward(st, p + h * d), z, cycles=3)
    lm = O.twogrid_loss(st, O.hypernet_forward(st, p - h * d), z, cycles=3)
    assert abs((lp - lm) / (2 * h) - g @ d) <= 1e-6 * abs(g @ d)


# ------------------------------------------------------------ adaptive training (Algorithm 2)
def test_transposed_kernels_are_the_matrix_transpose():
    n = 7
    W = np.random.default_rng(20).standard_normal((9, n, n))
    np.testing.assert_allclose(D.kernels_matrix(O.transpose_kernels(W)), D.kernels_matrix(W).T, rtol=0, atol=0)


def _level_kernels(st_c, seed):
    """Random smoothing kernels for every smoothed level of st_c's Galerkin hierarchy."""
    mg = O.Multigrid(st_c)
    rng = np.random.default_rng(seed)
    return [O.jacobi_kernels(mg.field(j)) * (1 + 0.2 * rng.standard_normal((9, mg.n(j), mg.n(j))))
            for j in range(mg.levels - 1)]


def test_vcycle_loss_with_an_exact_coarse_solve_is_the_two_grid_loss():
    n = 15
    st = O.const_field(n, O.q1_rotated_stencil(0.1, 0.7))
    W = O.jacobi_kernels(st) * (1 + 0.1 * np.random.default_rng(21).standard_normal((9, n, n)))
    z = np.random.default_rng(22).standard_normal((3, n, n))
    Ac = D.field_matrix(O.rap(st))
    exact = lambda r: np.linalg.solve(Ac, r.ravel()).reshape(r.shape)
    for k in (1, 2):
        l0, g0 = O.twogrid_loss(st, W, z, want_grad=True, cycles=k)
        l1, g1 = O.vcycle_loss(st, W, exact, exact, z, cycles=k, want_grad=True)
        assert abs(l1 - l0) <= 1e-12 * l0
        np.testing.assert_allclose(g1, g0, rtol=0, atol=1e-12 * np.abs(g0).max())


@pytest.mark.parametrize("cycles", [1, 2])
def test_vcycle_loss_matches_dense_operators(cycles):
    """E = S (I - P M P^T A) S with M the dense matrix of the coarse V-cycle (applied to unit
    vectors); the transposed-kernel cycle is M^T."""
    n = 15
    st = O.const_field(n, O.q1_rotated_stencil(0.03, 2.2))
    W = O.jacobi_kernels(st) * (1 + 0.1 * np.random.default_rng(23).standard_normal((9, n, n)))
    z = np.random.default_rng(24).standard_normal((3, n, n))
    st_c = O.rap(st)
    ker = _level_kernels(st_c, 25)
    fwd, adj = O.coarse_vcycle(st_c, ker), O.coarse_vcycle(st_c, ker, transpose=True)
    nc = st_c.shape[1]
    M = np.stack([fwd(np.eye(nc * nc)[i].reshape(nc, nc)).ravel() for i in range(nc * nc)], axis=1)
    MT = np.stack([adj(np.eye(nc * nc)[i].reshape(nc, nc)).ravel() for i in range(nc * nc)], axis=1)
    np.testing.assert_allclose(MT, M.T, rtol=0, atol=1e-12 * np.abs(M).max())
    A, H, P = D.field_matrix(st), D.kernels_matrix(W), D.prolongation(n)
    S = np.eye(n * n) - H @ A
    E = np.linalg.matrix_power(S @ (np.eye(n * n) - P @ M @ P.T @ A) @ S, cycles)
    want = np.mean([np.sum((E @ zi.ravel()) ** 2) / (n * n) for zi in z])
    assert abs(O.vcycle_loss(st, W, fwd, adj, z, cycles=cycles) - want) <= 1e-12 * want


def test_vcycle_loss_gradient_matches_finite_differences():
    n = 15
    rng = np.random.default_rng(26)
    st = O.const_field(n, O.q1_rotated_stencil(10 ** rng.uniform(-3, 0), rng.uniform(0, math.pi)))
    st_c = O.rap(st)
    ker = _level_kernels(st_c, 27)
    fwd, adj = O.coarse_vcycle(st_c, ker), O.coarse_vcycle(st_c, ker, transpose=True)
    p = rng.standard_normal(NP) * 0.2
    z = rng.standard_normal((2, n, n))
    loss, g = O.vcycle_cnn_loss_and_grad(st, p, fwd, adj, z, cycles=2)
    h = 1e-6
    for i in list(rng.choice(NP, 8, replace=False)) + [NP - 1]:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (O.vcycle_loss(st, O.hypernet_forward(st, pp), fwd, adj, z, cycles=2)
              - O.vcycle_loss(st, O.hypernet_forward(st, pm), fwd, adj, z, cycles=2)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g).max(), 1e-12), (i, fd, g[i])


# ------------------------------------------------------------ fully connected network
NFC = 81 * 40 + 40 * 40 + 40 * 40 + 40 * 9


def test_fc_parameter_count_is_the_papers():
    assert O.fc_nparams() == NFC == 6800


def test_fc_zero_last_layer_is_weighted_jacobi():
    n = 7
    st = O.const_field(n, O.q1_rotated_stencil(0.2, 0.3))
    p = np.random.default_rng(30).standard_normal(NFC)
    p[-360:] = 0.0
    np.testing.assert_allclose(O.fc_forward(st, p), O.jacobi_kernels(st), rtol=1e-15, atol=0)


def _torch_fc(st, p):
    """The same network in torch (float64): unfold of the normalised stencil field gives the
    3x3-neighbourhood features; linear layers and leaky_relu from torch.nn.functional."""
    n = st.shape[1]
    a0 = torch.from_numpy(st / st[4])[None]                      # [1, 9, n, n]
    U = F.unfold(a0, 3, padding=1)[0]                            # [9*9, n*n]: (c, ky, kx) major
    U = U.reshape(9, 9, n * n).permute(1, 0, 2).reshape(81, n * n)  # feature 9 m + c
    x = U.T
    pt = torch.from_numpy(p).requires_grad_(True)
    o = 0
    h = x
    for l, (co, ci) in enumerate([(40, 81), (40, 40), (40, 40), (9, 40)]):
        w = pt[o:o + co * ci].reshape(co, ci)
        o += co * ci
        h = F.linear(h, w)
        if l < 3:
            h = F.leaky_relu(h, 0.01)
    out = h.T.reshape(9, n, n)
    d = torch.from_numpy(st[4])
    W = out.clone()
    W[4] = W[4] + 2.0 / 3.0
    return W / d, pt


def test_fc_forward_and_backward_match_torch_autograd():
    n = 9
    rng = np.random.default_rng(31)
    st = O.varcoef5_field(n, np.exp(rng.standard_normal((n + 1, n + 1))))
    p = rng.standard_normal(NFC) * 0.1
    Wt, pt = _torch_fc(st, p)
    np.testing.assert_allclose(O.fc_forward(st, p), Wt.detach().numpy(), rtol=1e-12, atol=1e-14)
    dW = rng.standard_normal((9, n, n))
    (Wt * torch.from_numpy(dW)).sum().backward()
    np.testing.assert_allclose(O.fc_backward(st, p, dW), pt.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_fc_loss_gradient_matches_finite_differences():
    n = 15
    rng = np.random.default_rng(32)
    st = O.const_field(n, O.q1_rotated_stencil(0.05, 2.0))
    p = rng.standard_normal(NFC) * 0.05
    z = rng.standard_normal((2, n, n))
    _, g = O.fc_loss_and_grad(st, p, z)
    h = 1e-6
    for i in list(rng.choice(NFC, 8, replace=False)) + [NFC - 1, 0]:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (O.twogrid_loss(st, O.fc_forward(st, pp), z) - O.twogrid_loss(st, O.fc_forward(st, pm), z)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g).max(), 1e-12), (i, fd, g[i])
