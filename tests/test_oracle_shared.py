"""Pins of the shared-kernel network oracle (Sec. 6.2: 378 parameters).

The paper prints the count; the forward pass is checked against a layer-by-layer scipy
correlation of the summed input channels (sharing nothing with the C oracle's dense
convolution), the expansion and its gradient against each other by the adjoint identity,
and the loss gradient against central differences.
"""
import numpy as np
from scipy.signal import correlate2d

import oracle as O


def _field(n, seed):
    rng = np.random.default_rng(seed)
    return O.varcoef5_field(n, np.exp(rng.standard_normal((n + 1, n + 1)))) + \
        0.2 * O.paper9_field(n, rng.uniform(0.5, 2.0, (n + 1, n + 1)))


def test_parameter_count_is_the_papers():
    # Sec. 6.2: three convolutional layers of 7, 5 and 3 channels and a 27 x 9 layer, 378
    assert O.shared_nparams() == 378


def _corr(a, k):
    return correlate2d(a, k.reshape(3, 3), mode="same", boundary="fill", fillvalue=0.0)


def _leaky(z):
    return np.where(z > 0, z, 0.01 * z)


def test_forward_is_one_kernel_per_output_channel_on_the_summed_inputs():
    n = 9
    st = _field(n, 0)
    rng = np.random.default_rng(1)
    p = rng.standard_normal(378) * 0.4
    omega = 0.7
    a = [st[c] / st[4] for c in range(9)]  # input channel c: tap c over the point's diagonal
    o = 0
    for co in (7, 5, 3):
        s = sum(a)
        a = [_leaky(_corr(s, p[o + 9 * j:o + 9 * j + 9])) for j in range(co)]
        o += 9 * co
    wf = p[o:].reshape(9, 3, 9)  # tap t, input channel c, window position
    out = np.array([sum(_corr(a[c], wf[t, c]) for c in range(3)) for t in range(9)])
    out[4] += omega
    ref = out / st[4]
    np.testing.assert_allclose(O.shared_forward(st, p, omega), ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def test_expansion_and_gradient_sum_are_adjoint():
    rng = np.random.default_rng(2)
    p = rng.standard_normal(378)
    g = rng.standard_normal(O.hypernet_nparams())
    lhs = float(O.shared_to_dense(p) @ g)
    assert abs(lhs - float(p @ O.shared_grad(g))) <= 1e-12 * np.abs(g).sum() * np.abs(p).max()
    # the expansion ties w[o][c] = k_o: every input channel of a layer carries the same kernel
    w1 = O.shared_to_dense(p)[:567].reshape(7, 9, 9)
    assert np.array_equal(w1, np.broadcast_to(p[:63].reshape(7, 1, 9), (7, 9, 9)))


def test_loss_gradient_matches_central_differences():
    n = 15
    rng = np.random.default_rng(3)
    st = O.const_field(n, O.q1_rotated_stencil(0.05, 0.9))
    p = rng.standard_normal(378) * 0.3
    p[135:] *= 0.2  # a convergent smoother
    z = rng.standard_normal((2, n, n))
    _, g = O.shared_loss_and_grad(st, p, z)
    h = 1e-6
    idx = [0, 40, 62, 63, 100, 108, 134, 135, 377] + list(rng.choice(378, 6, replace=False))
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (O.shared_loss_and_grad(st, pp, z)[0] - O.shared_loss_and_grad(st, pm, z)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * np.abs(g).max(), (i, fd, g[i])
