"""FP64 oracle of the stencil-to-smoother network with a stack of k = 3 output kernels.

Test infrastructure only, like the rest of this package.  Plain PyTorch CPU operations in
float64; the gradient of the loss is PyTorch's reverse mode over those operations.

Sec. 4 maps each point's stencil neighbourhood to a stack of 3x3 convolution kernels
(Sec. 4.2: three kernels per point, Fig. convolution).  The network is the one of the
k = 1 oracle (9 input channels: the point's stencil over its diagonal; 3x3 convolutions
9 -> 7 -> 5 -> 3 with LeakyReLU(0.01) and zero padding; a layer from the 3x3 window of the
3-channel map) with 27 outputs instead of 9: out_1, out_2, out_3, one 3x3 kernel each.

Readings of the paper:
  - The three kernels act as a stack, H v = K3(K2(K1 v)), every K_k(u)(x) = sum_t
    K_k[t](x) u(x + d_t) with u zero outside the grid (a stack of convolutions, Sec. 4).
  - Scaling: K1 = (omega delta + out_1) / D, K2 = delta + out_2, K3 = delta + out_3
    (delta the identity kernel).  A zero last layer is weighted Jacobi, as for k = 1, and
    the stack reduces to the k = 1 network whenever out_2 = out_3 = 0.
Parameters: w1[7][9][3][3], w2[5][7][3][3], w3[3][5][3][3], wf[27][3][3][3] (row 9k + t
of wf: tap t of kernel k + 1): 1 746 values.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

from .oracle import _f64

NK = 3
SIZES = [(7, 9), (5, 7), (3, 5), (9 * NK, 3)]
NPARAMS = sum(co * ci * 9 for co, ci in SIZES)


def _t(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float64))


def _split(params: torch.Tensor):
    out, o = [], 0
    for co, ci in SIZES:
        out.append(params[o:o + co * ci * 9].reshape(co, ci, 3, 3))
        o += co * ci * 9
    return out


def network(st, params: torch.Tensor) -> torch.Tensor:
    """out [27, n, n] of the network on one stencil field st [9, n, n]."""
    st = _t(st)
    w1, w2, w3, wf = _split(params)
    a = (st / st[4]).unsqueeze(0)
    for w in (w1, w2, w3):
        z = F.conv2d(a, w, padding=1)
        a = torch.where(z > 0, z, 0.01 * z)
    return F.conv2d(a, wf, padding=1)[0]


def kernels(st, params: torch.Tensor, omega: float = 2.0 / 3.0) -> torch.Tensor:
    """The stack K [3, 9, n, n]: K1 = (omega delta + out_1)/D, K_k = delta + out_k (k = 2, 3)."""
    st = _t(st)
    out = network(st, params).reshape(NK, 9, *st.shape[1:])
    delta = torch.zeros(9, 1, 1, dtype=torch.float64)
    delta[4] = 1.0
    k1 = (omega * delta + out[0]) / st[4]
    return torch.stack([k1] + [delta + out[k] for k in range(1, NK)])


def _shift(v: torch.Tensor, di: int, dj: int) -> torch.Tensor:
    """u(x + (di, dj)) on the grid, zero where x + (di, dj) leaves it."""
    p = F.pad(v, (1, 1, 1, 1))
    n = v.shape[-1]
    return p[..., 1 + di:1 + di + n, 1 + dj:1 + dj + n]


def apply_kernel(K: torch.Tensor, v: torch.Tensor) -> torch.Tensor:
    """(K v)(x) = sum_t K[t](x) v(x + d_t), v zero outside the grid."""
    return sum(K[t] * _shift(v, t // 3 - 1, t % 3 - 1) for t in range(9))


def apply_kernel_T(K: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    """(K^T w)(y) = sum_t K[t](y - d_t) w(y - d_t)."""
    return sum(_shift(K[t] * w, -(t // 3 - 1), -(t % 3 - 1)) for t in range(9))


def apply_H(Ks: torch.Tensor, v: torch.Tensor) -> torch.Tensor:
    for K in Ks:
        v = apply_kernel(K, v)
    return v


def apply_HT(Ks: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    for K in reversed(list(Ks)):
        w = apply_kernel_T(K, w)
    return w


def apply_A(st, v: torch.Tensor) -> torch.Tensor:
    return apply_kernel(_t(st), v)


def restrict(r: torch.Tensor) -> torch.Tensor:
    """P^T r: coarse point I sits at fine 2I+1, weights 1/4 [1 2 1; 2 4 2; 1 2 1] x 4."""
    w = torch.tensor([[0.25, 0.5, 0.25], [0.5, 1.0, 0.5], [0.25, 0.5, 0.25]], dtype=torch.float64)
    return F.conv2d(r[None, None], w[None, None], stride=2)[0, 0]


def prolong(ec: torch.Tensor, n: int) -> torch.Tensor:
    """P e_c (bilinear): the transpose of restrict."""
    w = torch.tensor([[0.25, 0.5, 0.25], [0.5, 1.0, 0.5], [0.25, 0.5, 0.25]], dtype=torch.float64)
    return F.conv_transpose2d(ec[None, None], w[None, None], stride=2)[0, 0][:n, :n]


def coarse_vcycle(st_c, level_params, omega: float = 2.0 / 3.0):
    """Algorithm 2's coarse solve: M, one V(1,1) cycle from zero (Algorithm 1) of the
    Galerkin hierarchy of st_c, level l smoothed by the stack of network level_params[l]
    (the last set below that) on that level's own field, FP64 direct solve on the
    coarsest.  Returns M as a function of a torch right-hand side; it is linear in it, so
    the adjoint M^T of the loss gradient is what autograd takes through it."""
    from .oracle import dense_matrix, rap

    sts = [_f64(st_c)]
    while sts[-1].shape[1] > 3 and (sts[-1].shape[1] - 1) % 2 == 0:
        sts.append(rap(sts[-1]))
    sets = [_t(p) for p in level_params]
    with torch.no_grad():
        Ks = [kernels(s, sets[min(l, len(sets) - 1)], omega) for l, s in enumerate(sts[:-1])]
    Ac = torch.from_numpy(dense_matrix(sts[-1]))

    def level(l, f):
        n = sts[l].shape[1]
        if l == len(sts) - 1:
            return torch.linalg.solve(Ac, f.reshape(-1)).reshape(n, n)
        u = apply_H(Ks[l], f)                                   # pre-smoothing from u = 0
        uc = level(l + 1, restrict(f - apply_A(sts[l], u)))     # restriction, coarse cycle
        u = u + prolong(uc, n)                                  # prolongation
        return u + apply_H(Ks[l], f - apply_A(sts[l], u))       # post-smoothing

    return lambda rc: level(0, rc)


def loss(st, coarse_st, params: torch.Tensor, z, omega: float = 2.0 / 3.0, cycles: int = 1,
         coarse=None) -> torch.Tensor:
    """(1/Z) sum_j ||E^k z_j||^2 / n^2 with E = S C S, S = I - H A, C = I - P A_c^{-1} P^T A
    (Sec. 3.2, eq. twogrid; A_c = P^T A P is given as the coarse field coarse_st).  With
    `coarse` (a function of the coarse right-hand side, e.g. coarse_vcycle) A_c^{-1} is
    replaced by it: Algorithm 2's objective at one level."""
    st = _t(st)
    n = st.shape[-1]
    nc = (n - 1) // 2
    Ks = kernels(st, params, omega)
    Ac = _dense(coarse_st)
    total = torch.zeros((), dtype=torch.float64)
    z = _t(z)
    for zj in z:
        e = zj
        for _ in range(cycles):
            e = e - apply_H(Ks, apply_A(st, e))
            rc = restrict(apply_A(st, e))
            ec = coarse(rc) if coarse is not None else torch.linalg.solve(Ac, rc.reshape(-1)).reshape(nc, nc)
            e = e - prolong(ec, n)
            e = e - apply_H(Ks, apply_A(st, e))
        total = total + (e * e).sum()
    return total / (z.shape[0] * n * n)


def _dense(st) -> torch.Tensor:
    st = _t(st)
    n = st.shape[-1]
    A = torch.zeros(n * n, n * n, dtype=torch.float64)
    for t in range(9):
        di, dj = t // 3 - 1, t % 3 - 1
        for i in range(n):
            for j in range(n):
                ii, jj = i + di, j + dj
                if 0 <= ii < n and 0 <= jj < n:
                    A[i * n + j, ii * n + jj] = st[t, i, j]
    return A


def loss_and_grad(st, coarse_st, params, z, omega: float = 2.0 / 3.0, cycles: int = 1, coarse=None):
    p = _t(params).clone().requires_grad_(True)
    L = loss(st, coarse_st, p, z, omega, cycles, coarse)
    (g,) = torch.autograd.grad(L, p)
    return float(L.detach()), g.numpy()


def k1_params(params) -> np.ndarray:
    """The k = 1 network that the stack reduces to when out_2 = out_3 = 0: the same
    convolutions and the first nine rows of the last layer."""
    params = _f64(params)
    conv = sum(co * ci * 9 for co, ci in SIZES[:3])
    return np.concatenate([params[:conv], params[conv:conv + 9 * 27]])


class StackMultigrid:
    """Galerkin hierarchy of st0 (Algorithm 1, V(1,1)) smoothed on every level but the
    coarsest by the stack of the one network evaluated on that level's own stencil field."""

    def __init__(self, st0, params, omega: float = 2.0 / 3.0, coarsest_n: int = 3):
        from .oracle import dense_matrix, rap

        self.st = [_f64(st0)]
        while self.st[-1].shape[1] > coarsest_n and (self.st[-1].shape[1] - 1) % 2 == 0:
            self.st.append(rap(self.st[-1]))
        p = _t(params)
        with torch.no_grad():
            self.K = [kernels(s, p, omega) for s in self.st[:-1]]
        self.Ac = dense_matrix(self.st[-1])

    def _smooth(self, l, f, u):
        from .oracle import apply

        with torch.no_grad():
            h = apply_H(self.K[l], torch.from_numpy(f - apply(self.st[l], u))).numpy()
        return u + h

    def _level(self, l, f, u):
        from .oracle import apply, prolong, restrict

        u = self._smooth(l, f, u)
        rc = restrict(f - apply(self.st[l], u))
        if l + 1 == len(self.st) - 1:
            nc = rc.shape[0]
            uc = np.linalg.solve(self.Ac, rc.reshape(-1)).reshape(nc, nc)
        else:
            uc = self._level(l + 1, rc, np.zeros_like(rc))
        u = u + prolong(uc, self.st[l].shape[1])
        return self._smooth(l, f, u)

    def vcycle(self, b, x) -> np.ndarray:
        """One V(1,1) cycle of Algorithm 1 on A x = b from the iterate x."""
        return self._level(0, _f64(b), _f64(x).copy())

    def solve(self, b, rtol: float = 1e-8, max_cycles: int = 1000):
        """V-cycles from x = 0 until ||b - A x|| / ||b|| < rtol; (x, hist)."""
        from .oracle import apply

        b = _f64(b)
        x = np.zeros_like(b)
        bn = np.linalg.norm(b)
        hist = [1.0]
        while len(hist) - 1 < max_cycles and not hist[-1] < rtol:
            x = self._level(0, b, x)
            hist.append(np.linalg.norm(b - apply(self.st[0], x)) / bn)
        return x, np.array(hist)
