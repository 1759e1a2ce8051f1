"""FP64 oracle of the shared-kernel linear smoother of Sec. 6 (eq. full-coarsening-smoother).

Test infrastructure only, like the rest of this package.

On level l the smoother is a fixed linear map built from six 3x3 kernels phi_1 .. phi_6,
shared by every grid point:

    H v = f_5(f_4(f_3(f_2(f_1(v))))) + f_6(v),   f_k(u)(x) = sum_t phi_k[t] u(x + d_t),

with the tap convention of every other smoother here (t = 3*(di+1) + (dj+1), row = y) and
each layer's output defined on the n x n interior only: its input is taken as zero outside
the grid (the Dirichlet exterior), so near the boundary the chain is not one wide stencil.
The map is linear in v (no activation: Sec. 6 uses the linear network to read the kernels
as smoothers, Sec. 5).  Parameters of one level: phi[6][9] = (phi_1 .. phi_5, phi_6).

Readings of the paper:
  - Sec. 6 initialises phi_1 .. phi_5 with zeros and phi_6 with the inverse Jacobi stencil.
    With all five chain kernels zero every gradient of the chain vanishes (each one is a
    product of the other four), so training would never move them.  Here phi_1 .. phi_4
    start as the identity kernel (centre tap 1) and phi_5 at zero: H is still exactly
    weighted Jacobi at the start, and phi_5 receives a gradient from the first step.
  - The multigrid cycle is Algorithm 1 with nu1 = nu2 = 1, the same as for every other
    smoother: u += H (f - A u) before and after the coarse correction.
"""
from __future__ import annotations

import numpy as np

from .oracle import _f64, apply, dense_matrix, prolong, rap, restrict

NPHI = 6  # kernels per level: the chain f_1 .. f_5, then the parallel f_6
NLIN = NPHI * 9


def _taps():
    return [(t // 3 - 1, t % 3 - 1) for t in range(9)]


def conv(phi, v) -> np.ndarray:
    """f(v)(x) = sum_t phi[t] v(x + d_t), v zero outside the n x n grid."""
    v = _f64(v)
    n = v.shape[0]
    y = np.zeros_like(v)
    for t, (di, dj) in enumerate(_taps()):
        i0, i1 = max(0, -di), min(n, n - di)
        j0, j1 = max(0, -dj), min(n, n - dj)
        y[i0:i1, j0:j1] += phi[t] * v[i0 + di:i1 + di, j0 + dj:j1 + dj]
    return y


def conv_T(phi, v) -> np.ndarray:
    """Transpose of conv(phi, .): (f^T w)(y) = sum_t phi[t] w(y - d_t)."""
    v = _f64(v)
    n = v.shape[0]
    y = np.zeros_like(v)
    for t, (di, dj) in enumerate(_taps()):
        i0, i1 = max(0, di), min(n, n + di)
        j0, j1 = max(0, dj), min(n, n + dj)
        y[i0:i1, j0:j1] += phi[t] * v[i0 - di:i1 - di, j0 - dj:j1 - dj]
    return y


def chain_forward(phi, v):
    """Intermediate maps w_0 = v, w_k = f_k(w_{k-1}) (k = 1..4) and H v."""
    phi = _f64(phi).reshape(NPHI, 9)
    w = [_f64(v)]
    for k in range(4):
        w.append(conv(phi[k], w[-1]))
    return w, conv(phi[4], w[4]) + conv(phi[5], w[0])


def apply_H(phi, v) -> np.ndarray:
    return chain_forward(phi, v)[1]


def apply_HT(phi, v) -> np.ndarray:
    """H^T v = f_1^T(f_2^T(f_3^T(f_4^T(f_5^T v)))) + f_6^T v."""
    phi = _f64(phi).reshape(NPHI, 9)
    v = _f64(v)
    g = conv_T(phi[4], v)
    for k in (3, 2, 1, 0):
        g = conv_T(phi[k], g)
    return g + conv_T(phi[5], v)


def _corr(g, u) -> np.ndarray:
    """D[t] = sum_x g(x) u(x + d_t) (u zero outside): the kernel gradient of conv(., u)."""
    n = g.shape[0]
    D = np.zeros(9)
    for t, (di, dj) in enumerate(_taps()):
        i0, i1 = max(0, -di), min(n, n - di)
        j0, j1 = max(0, -dj), min(n, n - dj)
        D[t] = np.sum(g[i0:i1, j0:j1] * u[i0 + di:i1 + di, j0 + dj:j1 + dj])
    return D


def grad_H(phi, v, g) -> np.ndarray:
    """d <g, H v> / d phi, shape [6][9] (reverse pass through the chain)."""
    phi = _f64(phi).reshape(NPHI, 9)
    w, _ = chain_forward(phi, v)
    d = np.zeros((NPHI, 9))
    d[5] = _corr(g, w[0])
    lam = _f64(g)
    for k in (4, 3, 2, 1, 0):
        d[k] = _corr(lam, w[k])
        if k > 0:
            lam = conv_T(phi[k], lam)
    return d


def jacobi_params(d: float, omega: float = 2.0 / 3.0) -> np.ndarray:
    """The starting point of training: H = omega / d (phi_1..4 identity, phi_5 zero)."""
    phi = np.zeros((NPHI, 9))
    phi[0:4, 4] = 1.0
    phi[5, 4] = omega / d
    return phi


def transpose_params(phi) -> np.ndarray:
    """Parameters of H^T as a chain of the same form: the chain in reverse order with every
    kernel mirrored (f^T is conv with phi[8 - t])."""
    phi = _f64(phi).reshape(NPHI, 9)
    out = np.empty_like(phi)
    for k in range(5):
        out[k] = phi[4 - k][::-1]
    out[5] = phi[5][::-1]
    return out


# ------------------------------------------------------------------ multigrid (Algorithm 1)
class LinearMultigrid:
    """Galerkin hierarchy of st0 with the shared-kernel linear smoother on every level but
    the coarsest; phis[l] (or phis[-1] for deeper levels) smooths level l."""

    def __init__(self, st0, phis, coarsest_n: int = 3, nu1: int = 1, nu2: int = 1):
        """nu1, nu2: the smoothing steps before and after the coarse correction."""
        self.nu1, self.nu2 = nu1, nu2
        self.st = [_f64(st0)]
        while self.st[-1].shape[1] > coarsest_n and (self.st[-1].shape[1] - 1) % 2 == 0:
            self.st.append(rap(self.st[-1]))
        self.L = len(self.st)
        phis = [_f64(p).reshape(NPHI, 9) for p in phis]
        self.phi = [phis[min(l, len(phis) - 1)] for l in range(self.L)]
        self.Ac = dense_matrix(self.st[-1])

    def n(self, level: int) -> int:
        return self.st[level].shape[1]

    def _smooth(self, l, f, u):
        return u + apply_H(self.phi[l], f - apply(self.st[l], u))

    def _level(self, l, f, u):
        for _ in range(self.nu1):                          # pre-smoothing
            u = self._smooth(l, f, u)
        rc = restrict(f - apply(self.st[l], u))            # r^(l+1) = P^T (f - A u)
        if l + 1 == self.L - 1:
            nc = self.n(l + 1)
            uc = np.linalg.solve(self.Ac, rc.reshape(-1)).reshape(nc, nc)
        else:
            uc = self._level(l + 1, rc, np.zeros_like(rc))
        u = u + prolong(uc, self.n(l))                     # u += P u^(l+1)
        for _ in range(self.nu2):                          # post-smoothing
            u = self._smooth(l, f, u)
        return u

    def vcycle(self, b, x) -> np.ndarray:
        b, x = _f64(b), _f64(x)
        if self.L == 1:
            n = self.n(0)
            return np.linalg.solve(self.Ac, b.reshape(-1)).reshape(n, n)
        return self._level(0, b, x)

    def solve(self, b, x0=None, rtol: float = 1e-8, max_cycles: int = 1000):
        """V-cycles until ||b - A x|| / ||b|| < rtol; returns (x, hist), hist[k] after k cycles."""
        b = _f64(b)
        x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
        bn = np.linalg.norm(b)
        hist = [np.linalg.norm(b - apply(self.st[0], x)) / bn]
        while len(hist) - 1 < max_cycles and not hist[-1] < rtol:
            x = self.vcycle(b, x)
            hist.append(np.linalg.norm(b - apply(self.st[0], x)) / bn)
        return x, np.array(hist)


def coarse_vcycle(st_c, phis, transpose: bool = False):
    """r -> one V(1,1) cycle from zero on the hierarchy of st_c with the given per-level
    linear smoothers (transposed on every level when transpose is set)."""
    if transpose:
        phis = [transpose_params(p) for p in phis]
    mg = LinearMultigrid(st_c, phis)
    return lambda r: mg.vcycle(r, np.zeros_like(_f64(r)))


# ------------------------------------------------------------------ loss and its gradient
def loss_and_grad(st, phi, z, cycles: int = 1, coarse=None, coarse_t=None, want_grad: bool = True):
    """(1/Z) sum_j ||E^k z_j||^2 / n^2 with E = S C S, S = I - H A (Sec. 3.2, eq. twogrid) and
    dLoss/dphi [6][9].  C = I - P M P^T A: M = (P^T A P)^{-1} (the two-grid objective) when
    coarse is None, else M = coarse (one V-cycle of the trained hierarchy below, Algorithm 2)
    with its transpose coarse_t."""
    st, z = _f64(st), _f64(z)
    phi = _f64(phi).reshape(NPHI, 9)
    n = st.shape[1]
    nz = z.shape[0]
    if coarse is None:
        Ac = dense_matrix(rap(st))
        nc = (n - 1) // 2

        def coarse(r):
            return np.linalg.solve(Ac, r.reshape(-1)).reshape(nc, nc)

        coarse_t = coarse  # A_c is symmetric
    dphi = np.zeros((NPHI, 9))
    loss = 0.0
    for zj in z:
        e = zj.copy()
        V0, V2 = [], []
        for _ in range(cycles):
            v0 = apply(st, e)
            e1 = e - apply_H(phi, v0)
            e2 = e1 - prolong(coarse(restrict(apply(st, e1))), n)
            v2 = apply(st, e2)
            e = e2 - apply_H(phi, v2)
            V0.append(v0)
            V2.append(v2)
        loss += np.sum(e * e) / (nz * n * n)
        if not want_grad:
            continue
        g = 2.0 * e / (nz * n * n)
        for c in range(cycles - 1, -1, -1):
            dphi -= grad_H(phi, V2[c], g)                  # e3 = e2 - H v2
            g = g - apply(st, apply_HT(phi, g))
            g = g - apply(st, prolong(coarse_t(restrict(g)), n))
            dphi -= grad_H(phi, V0[c], g)                  # e1 = e0 - H v0
            if c > 0:
                g = g - apply(st, apply_HT(phi, g))
    return (loss, dphi) if want_grad else loss
