"""ctypes front end of the FP64 C oracle (mg_oracle.c).

Test infrastructure only (see the package docstring).  Every function takes and
returns numpy float64 arrays; grids are ``[n, n]`` with row index = y, column = x,
and stencil fields / per-point kernels are ``[9, n, n]`` with tap k = 3*(di+1)+(dj+1).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_D = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, -O2, no machine-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mg_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.or_mg_create.restype = ctypes.c_void_p
        L.or_mg_create.argtypes = [ctypes.c_int, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        for name in ("or_mg_destroy",):
            getattr(L, name).argtypes = [ctypes.c_void_p]
        L.or_mg_levels.argtypes = [ctypes.c_void_p]
        L.or_mg_n.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_mg_get_field.argtypes = [ctypes.c_void_p, ctypes.c_int, _D]
        L.or_mg_get_kernels.argtypes = [ctypes.c_void_p, ctypes.c_int, _D]
        L.or_mg_set_kernels.argtypes = [ctypes.c_void_p, ctypes.c_int, _D]
        L.or_mg_set_jacobi.argtypes = [ctypes.c_void_p, ctypes.c_double]
        L.or_mg_set_cnn.argtypes = [ctypes.c_void_p, _D, ctypes.c_double, ctypes.c_int]
        L.or_mg_vcycle.argtypes = [ctypes.c_void_p, _D, _D]
        L.or_mg_solve.argtypes = [ctypes.c_void_p, _D, _D, ctypes.c_double, ctypes.c_int, _D]
        L.or_bf16.restype = ctypes.c_double
        L.or_bf16.argtypes = [ctypes.c_double]
        L.or_twogrid_loss.restype = ctypes.c_double
        L.or_twogrid_loss.argtypes = [ctypes.c_int, _D, _D, ctypes.c_int, _D, _D]
        L.or_twogrid_loss_k.restype = ctypes.c_double
        L.or_twogrid_loss_k.argtypes = [ctypes.c_int, _D, _D, ctypes.c_int, _D, ctypes.c_int, _D]
        L.or_cholesky.argtypes = [ctypes.c_int, _D]
        L.or_cholesky_solve.argtypes = [ctypes.c_int, _D, _D]
        L.or_q1_rotated_stencil.argtypes = [ctypes.c_double, ctypes.c_double, _D]
        L.or_fd_rotated_stencil.argtypes = [ctypes.c_double, ctypes.c_double, _D]
        L.or_hypernet_forward.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_int, _D]
        L.or_hypernet_backward.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_int, _D, _D]
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------- discretisations
def q1_rotated_stencil(eps: float, theta: float) -> np.ndarray:
    s = np.zeros(9)
    lib().or_q1_rotated_stencil(float(eps), float(theta), _p(s))
    return s.reshape(3, 3)


def fd_rotated_stencil(xi: float, theta: float) -> np.ndarray:
    s = np.zeros(9)
    lib().or_fd_rotated_stencil(float(xi), float(theta), _p(s))
    return s.reshape(3, 3)


def fe_q1_field(n: int, kxx, kxy, kyy) -> np.ndarray:
    """Q1 field; kxx/kxy/kyy scalars (constant tensor) or [(n+1),(n+1)] cell arrays."""
    per_cell = int(np.ndim(kxx) > 0)
    kxx, kxy, kyy = (_f64(np.atleast_1d(v)) for v in (kxx, kxy, kyy))
    st = np.zeros((9, n, n))
    lib().or_fe_q1_field(n, _p(kxx), _p(kxy), _p(kyy), per_cell, _p(st))
    return st


def paper9_field(n: int, g_cells) -> np.ndarray:
    g = _f64(g_cells)
    assert g.shape == (n + 1, n + 1)
    st = np.zeros((9, n, n))
    lib().or_paper9_field(n, _p(g), _p(st))
    return st


def varcoef5_field(n: int, a_cells) -> np.ndarray:
    a = _f64(a_cells)
    assert a.shape == (n + 1, n + 1)
    st = np.zeros((9, n, n))
    lib().or_varcoef5_field(n, _p(a), _p(st))
    return st


def const_field(n: int, s) -> np.ndarray:
    s = _f64(np.asarray(s).reshape(9))
    st = np.zeros((9, n, n))
    lib().or_const_field(n, _p(s), _p(st))
    return st


# ---------------------------------------------------------------- operators
def apply(st: np.ndarray, x) -> np.ndarray:
    n = st.shape[1]
    st, x = _f64(st), _f64(x)
    y = np.zeros((n, n))
    lib().or_apply(n, _p(st), _p(x), _p(y))
    return y


def restrict(r) -> np.ndarray:
    r = _f64(r)
    n = r.shape[0]
    rc = np.zeros(((n - 1) // 2, (n - 1) // 2))
    lib().or_restrict(n, _p(r), _p(rc))
    return rc


def prolong(ec, n: int) -> np.ndarray:
    ec = _f64(ec)
    e = np.zeros((n, n))
    lib().or_prolong_add(n, _p(ec), _p(e))
    return e


def rap(st) -> np.ndarray:
    st = _f64(st)
    n = st.shape[1]
    nc = (n - 1) // 2
    stc = np.zeros((9, nc, nc))
    lib().or_rap(n, _p(st), _p(stc))
    return stc


def dense_matrix(st) -> np.ndarray:
    st = _f64(st)
    n = st.shape[1]
    A = np.zeros((n * n, n * n))
    lib().or_dense_matrix(n, _p(st), _p(A))
    return A


# ---------------------------------------------------------------- smoothers
def jacobi_kernels(st, omega: float = 2.0 / 3.0) -> np.ndarray:
    st = _f64(st)
    n = st.shape[1]
    W = np.zeros((9, n, n))
    lib().or_jacobi_kernels(n, _p(st), ctypes.c_double(omega), _p(W))
    return W


def apply_H(W, v) -> np.ndarray:
    W, v = _f64(W), _f64(v)
    n = v.shape[0]
    y = np.zeros((n, n))
    lib().or_apply_H(n, _p(W), _p(v), _p(y))
    return y


def apply_HT(W, v) -> np.ndarray:
    W, v = _f64(W), _f64(v)
    n = v.shape[0]
    y = np.zeros((n, n))
    lib().or_apply_HT(n, _p(W), _p(v), _p(y))
    return y


def smooth(st, W, f, u, nsteps: int = 1) -> np.ndarray:
    st, W, f = _f64(st), _f64(W), _f64(f)
    u = _f64(u).copy()
    n = st.shape[1]
    lib().or_smooth(n, _p(st), _p(W), _p(f), _p(u), nsteps)
    return u


def gauss_seidel(st, f, u) -> np.ndarray:
    st, f = _f64(st), _f64(f)
    u = _f64(u).copy()
    lib().or_gauss_seidel(st.shape[1], _p(st), _p(f), _p(u))
    return u


def bf16(v: float) -> float:
    return lib().or_bf16(float(v))


# ---------------------------------------------------------------- multigrid
class Multigrid:
    """Galerkin hierarchy + V-cycle (Algorithm 1) + solve, all FP64."""

    def __init__(self, st0, coarsest_n: int = 3, nu1: int = 1, nu2: int = 1):
        st0 = _f64(st0)
        self.h = lib().or_mg_create(st0.shape[1], _p(st0), coarsest_n, nu1, nu2)
        if not self.h:
            raise ValueError("coarsest operator is not SPD")

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_mg_destroy(self.h)
            self.h = None

    @property
    def levels(self) -> int:
        return lib().or_mg_levels(self.h)

    def n(self, level: int) -> int:
        return lib().or_mg_n(self.h, level)

    def field(self, level: int) -> np.ndarray:
        n = self.n(level)
        st = np.zeros((9, n, n))
        lib().or_mg_get_field(self.h, level, _p(st))
        return st

    def kernels(self, level: int) -> np.ndarray:
        n = self.n(level)
        W = np.zeros((9, n, n))
        lib().or_mg_get_kernels(self.h, level, _p(W))
        return W

    def set_kernels(self, level: int, W) -> None:
        W = _f64(W)
        lib().or_mg_set_kernels(self.h, level, _p(W))

    def set_jacobi(self, omega: float = 2.0 / 3.0) -> None:
        lib().or_mg_set_jacobi(self.h, ctypes.c_double(omega))

    def set_cnn(self, params, omega: float = 2.0 / 3.0, bf16: bool = False) -> None:
        params = _f64(params)
        assert params.size == hypernet_nparams()
        lib().or_mg_set_cnn(self.h, _p(params), ctypes.c_double(omega), int(bf16))

    def vcycle(self, b, x) -> np.ndarray:
        b = _f64(b)
        x = _f64(x).copy()
        lib().or_mg_vcycle(self.h, _p(b), _p(x))
        return x

    def solve(self, b, x0=None, rtol: float = 1e-8, max_cycles: int = 1000):
        b = _f64(b)
        x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
        hist = np.zeros(max_cycles + 1)
        k = lib().or_mg_solve(self.h, _p(b), _p(x), ctypes.c_double(rtol), max_cycles, _p(hist))
        return x, hist[: k + 1]


# ---------------------------------------------------------------- network + loss
def hypernet_nparams() -> int:
    return lib().or_hypernet_nparams()


def hypernet_forward(st, params, omega: float = 2.0 / 3.0, bf16: bool = False) -> np.ndarray:
    st, params = _f64(st), _f64(params)
    n = st.shape[1]
    W = np.zeros((9, n, n))
    lib().or_hypernet_forward(n, _p(st), _p(params), ctypes.c_double(omega), int(bf16), _p(W))
    return W


def hypernet_backward(st, params, dW, omega: float = 2.0 / 3.0, bf16: bool = False) -> np.ndarray:
    st, params, dW = _f64(st), _f64(params), _f64(dW)
    n = st.shape[1]
    g = np.zeros(params.size)
    lib().or_hypernet_backward(n, _p(st), _p(params), ctypes.c_double(omega), int(bf16), _p(dW), _p(g))
    return g


def twogrid_loss(st, W, z, want_grad: bool = False, cycles: int = 1):
    """Loss (1/Z) sum_j ||(S C S)^k z_j||^2 / n^2 (k = cycles) and, optionally, dLoss/dW.
    cycles = 1 is the two-grid objective of eq. twogrid; k > 1 the k-cycle form of eq.
    overalltrain that Algorithm 2 minimises."""
    st, W, z = _f64(st), _f64(W), _f64(z)
    n = st.shape[1]
    nz = z.shape[0]
    dW = np.zeros((9, n, n)) if want_grad else None
    if cycles == 1:
        loss = lib().or_twogrid_loss(n, _p(st), _p(W), nz, _p(z), _p(dW) if want_grad else None)
    else:
        loss = lib().or_twogrid_loss_k(n, _p(st), _p(W), nz, _p(z), int(cycles), _p(dW) if want_grad else None)
    return (loss, dW) if want_grad else loss


def cnn_loss_and_grad(st, params, z, omega: float = 2.0 / 3.0, bf16: bool = False, cycles: int = 1):
    """Loss of one problem as a function of the network parameters, with its gradient."""
    W = hypernet_forward(st, params, omega, bf16)
    loss, dW = twogrid_loss(st, W, z, want_grad=True, cycles=cycles)
    return loss, hypernet_backward(st, params, dW, omega, bf16)


# ------------------------------------------------ the shared-kernel network (Sec. 6.2)
# Sec. 6.2 counts 378 parameters for the convolutional network with 7, 5 and 3 channels and
# a 27 x 9 last layer: (7 + 5 + 3) * 9 + 27 * 9, one 3x3 kernel per output channel of each
# convolution.  Reading: that kernel acts on every input channel of its layer, out_o =
# k_o * (sum_c in_c).  This is the dense network with w[o][c] = k_o for every c, so the
# forward is the dense one on the expanded parameters, and by the chain rule the gradient
# of k_o is the sum over c of the dense gradient of w[o][c].
SHARED_CONV = ((7, 9), (5, 7), (3, 5))  # (output, input) channels of the convolutions


def shared_nparams() -> int:
    return sum(co * 9 for co, _ in SHARED_CONV) + 9 * 27


def shared_to_dense(params) -> np.ndarray:
    """k1[7][9], k2[5][9], k3[3][9], wf[243] -> w1[7][9][9], w2[5][7][9], w3[3][5][9], wf."""
    params = _f64(params)
    assert params.size == shared_nparams()
    out, o = [], 0
    for co, ci in SHARED_CONV:
        k = params[o:o + co * 9].reshape(co, 1, 9)
        out.append(np.broadcast_to(k, (co, ci, 9)).reshape(-1))
        o += co * 9
    out.append(params[o:])
    return np.concatenate(out)


def shared_grad(dense_grad) -> np.ndarray:
    """The gradient of the shared parameters from that of the expanded dense ones."""
    g = _f64(dense_grad)
    out, o = [], 0
    for co, ci in SHARED_CONV:
        out.append(g[o:o + co * ci * 9].reshape(co, ci, 9).sum(axis=1).reshape(-1))
        o += co * ci * 9
    out.append(g[o:])
    return np.concatenate(out)


def shared_forward(st, params, omega: float = 2.0 / 3.0, bf16: bool = False) -> np.ndarray:
    return hypernet_forward(st, shared_to_dense(params), omega, bf16)


def shared_loss_and_grad(st, params, z, omega: float = 2.0 / 3.0, bf16: bool = False, cycles: int = 1):
    loss, g = cnn_loss_and_grad(st, shared_to_dense(params), z, omega, bf16, cycles)
    return loss, shared_grad(g)


# ------------------------------------------------ adaptive (level-by-level) training
def transpose_kernels(W) -> np.ndarray:
    """Per-point kernels of H^T.  (H v)(x) = sum_k W_x[k] v(x + d_k), so
    (H^T v)(y) = sum_k W_{y - d_k}[k] v(y - d_k); as kernels at y with the offset
    d_{8-k} = -d_k: WT[k][y] = W[8 - k][y + d_k], zero where y + d_k leaves the grid."""
    W = _f64(W)
    n = W.shape[1]
    WT = np.zeros_like(W)
    for k in range(9):
        di, dj = k // 3 - 1, k % 3 - 1
        i0, i1 = max(0, -di), min(n, n - di)
        j0, j1 = max(0, -dj), min(n, n - dj)
        WT[k, i0:i1, j0:j1] = W[8 - k, i0 + di:i1 + di, j0 + dj:j1 + dj]
    return WT


def _shift_outer(g, v, n):
    """D[k][x] = g(x) v(x + d_k) (zero outside the grid): the weight gradient of H v."""
    D = np.zeros((9, n, n))
    for k in range(9):
        di, dj = k // 3 - 1, k % 3 - 1
        i0, i1 = max(0, -di), min(n, n - di)
        j0, j1 = max(0, -dj), min(n, n - dj)
        D[k, i0:i1, j0:j1] = g[i0:i1, j0:j1] * v[i0 + di:i1 + di, j0 + dj:j1 + dj]
    return D


def vcycle_loss(st, W, coarse, coarse_t, z, cycles: int = 1, want_grad: bool = False):
    """The objective Algorithm 2 minimises at one level l: the two-grid error propagation
    E = S (I - P M P^T A) S with S = I - H A, whose coarse solve is replaced by M, one
    V-cycle of the hierarchy below (already trained); loss = (1/Z) sum_j ||E^k z_j||^2 / n^2.
    coarse(r) applies M to a coarse vector, coarse_t(r) its transpose (the same V-cycle
    with transposed smoothing kernels on every level).  Optionally dLoss/dW: the adjoint
    runs the k cycles in reverse, C^T = I - A P M^T P^T."""
    st, W, z = _f64(st), _f64(W), _f64(z)
    n = st.shape[1]
    nz = z.shape[0]
    dW = np.zeros((9, n, n)) if want_grad else None
    loss = 0.0
    for zj in z:
        e = zj.copy()
        V0, V2 = [], []
        for _ in range(cycles):
            v0 = apply(st, e)                               # pre-smoothing e1 = e - H A e
            e1 = e - apply_H(W, v0)
            xc = coarse(restrict(apply(st, e1)))            # e2 = e1 - P M P^T A e1
            e2 = e1 - prolong(xc, n)
            v2 = apply(st, e2)                              # post-smoothing e = e2 - H A e2
            e = e2 - apply_H(W, v2)
            V0.append(v0)
            V2.append(v2)
        loss += np.sum(e * e) / (nz * n * n)
        if not want_grad:
            continue
        g = 2.0 * e / (nz * n * n)
        for c in range(cycles - 1, -1, -1):
            dW -= _shift_outer(g, V2[c], n)
            g = g - apply(st, apply_HT(W, g))
            g = g - apply(st, prolong(coarse_t(restrict(g)), n))
            dW -= _shift_outer(g, V0[c], n)
            if c > 0:
                g = g - apply(st, apply_HT(W, g))
    return (loss, dW) if want_grad else loss


def coarse_vcycle(st_c, kernels, transpose: bool = False):
    """r -> one V(1,1) cycle from zero on the Galerkin hierarchy of st_c, with the given
    per-level smoothing kernels (kernels[j] on level j of that hierarchy; transposed when
    transpose is set), coarsest level solved exactly."""
    mg = Multigrid(st_c)
    for j, W in enumerate(kernels):
        mg.set_kernels(j, transpose_kernels(W) if transpose else W)
    return lambda r: mg.vcycle(r, np.zeros_like(_f64(r)))


def vcycle_cnn_loss_and_grad(st, params, coarse, coarse_t, z, cycles: int = 1, omega: float = 2.0 / 3.0,
                             bf16: bool = False):
    """vcycle_loss as a function of the network parameters of this level, with its gradient."""
    W = hypernet_forward(st, params, omega, bf16)
    loss, dW = vcycle_loss(st, W, coarse, coarse_t, z, cycles, want_grad=True)
    return loss, hypernet_backward(st, params, dW, omega, bf16)


# ------------------------------------------------------------------- FGMRES (Sec. 6.4)
def fgmres(apply_A, precond, b, x0=None, restart: int = 30, rtol: float = 1e-6, max_iters: int = 500):
    """Right-preconditioned flexible GMRES(restart) (Sec. 6.4: multigrid as the
    preconditioner; flexible because a network smoother need not be a fixed linear map).
    Arnoldi on A M with the preconditioned directions z_j = M(v_j) kept, classical
    Gram-Schmidt with one re-orthogonalisation, Givens rotations on the Hessenberg
    matrix, x = x0 + Z y.  Stops when ||b - A x|| / ||b|| < rtol (the rotated least-squares
    residual, which equals the true one in exact arithmetic).
    Returns (x, history of relative residuals, iterations)."""
    b = _f64(b)
    shape = b.shape
    bv = b.ravel()
    x = np.zeros_like(bv) if x0 is None else _f64(x0).ravel().copy()
    A = lambda v: _f64(apply_A(v.reshape(shape))).ravel()
    M = lambda v: _f64(precond(v.reshape(shape))).ravel()
    bnorm = np.linalg.norm(bv)
    r = bv - A(x)
    hist = [np.linalg.norm(r) / bnorm]
    its = 0
    while hist[-1] >= rtol and its < max_iters:
        beta = np.linalg.norm(r)
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        j = 0
        while j < restart and its < max_iters:
            z = M(V[j])
            Z.append(z)
            w = A(z)
            h = np.array([vi @ w for vi in V])
            w = w - sum(hi * vi for hi, vi in zip(h, V))
            h2 = np.array([vi @ w for vi in V])           # second Gram-Schmidt pass
            w = w - sum(hi * vi for hi, vi in zip(h2, V))
            H[: j + 1, j] = h + h2
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j])
            for i in range(j):                             # earlier rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rho = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / rho, H[j + 1, j] / rho
            H[j, j], H[j + 1, j] = rho, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            j += 1
            its += 1
            hist.append(abs(g[j]) / bnorm)
            if hist[-1] < rtol:
                break
        y = np.linalg.solve(np.triu(H[:j, :j]), g[:j])
        x = x + sum(yi * zi for yi, zi in zip(y, Z))
        r = bv - A(x)
    return x.reshape(shape), np.array(hist), its


# ------------------------------------------- fully connected stencil-to-smoother network
FC_LAYERS = [(40, 81), (40, 40), (40, 40), (9, 40)]  # (out, in): "4 fully connected layers" of Sec. 6.2
FC_SLOPE = 0.01


def fc_nparams() -> int:
    return sum(o * i for o, i in FC_LAYERS)


def _bf16_array(a):
    return np.vectorize(bf16)(a) if a.size else a


def fc_features(st, bf16_round: bool = False) -> np.ndarray:
    """Sec. 4.2 (parameterisation with fully connected layers): the representation of a grid
    point is the 81 stencil values of its 3x3 neighbourhood.  Feature 9 m + c is tap c of the
    neighbour at offset d_m (m = 3 (di + 1) + (dj + 1)), divided by that neighbour's own
    diagonal (the input normalisation of the convolutional network); zero outside the grid.
    Returns [n*n, 81]."""
    st = _f64(st)
    n = st.shape[1]
    a0 = st / st[4]
    if bf16_round:
        a0 = _bf16_array(a0)
    X = np.zeros((n, n, 81))
    for m in range(9):
        di, dj = m // 3 - 1, m % 3 - 1
        i0, i1 = max(0, -di), min(n, n - di)
        j0, j1 = max(0, -dj), min(n, n - dj)
        X[i0:i1, j0:j1, 9 * m:9 * m + 9] = np.moveaxis(a0[:, i0 + di:i1 + di, j0 + dj:j1 + dj], 0, -1)
    return X.reshape(n * n, 81)


def _fc_weights(params, bf16_round):
    params = _f64(params)
    assert params.size == fc_nparams()
    out, o = [], 0
    for co, ci in FC_LAYERS:
        w = params[o:o + co * ci].reshape(co, ci)
        out.append(_bf16_array(w) if bf16_round else w)
        o += co * ci
    return out


def fc_forward(st, params, omega: float = 2.0 / 3.0, bf16: bool = False) -> np.ndarray:
    """Per-point kernels W = (omega delta_4 + NN)/D from the fully connected network
    81 -> 40 -> 40 -> 40 -> 9, LeakyReLU(0.01) after the hidden layers, no biases (6 800
    parameters, Sec. 6.2); with bf16, weights, inputs and activations rounded to bfloat16."""
    st = _f64(st)
    n = st.shape[1]
    Ws = _fc_weights(params, bf16)
    a = fc_features(st, bf16)
    for l, w in enumerate(Ws):
        z = a @ w.T
        if l < 3:
            a = np.where(z > 0, z, FC_SLOPE * z)
            if bf16:
                a = _bf16_array(a)
        else:
            a = z
    out = a.T.reshape(9, n, n)
    W = out.copy()
    W[4] += omega
    return W / st[4]


def fc_backward(st, params, dW, omega: float = 2.0 / 3.0, bf16: bool = False) -> np.ndarray:
    """dLoss/dparams of fc_forward given dLoss/dW (rounding treated as the identity)."""
    st, dW = _f64(st), _f64(dW)
    n = st.shape[1]
    Ws = _fc_weights(params, bf16)
    acts, zs = [fc_features(st, bf16)], []
    for l, w in enumerate(Ws):
        z = acts[-1] @ w.T
        zs.append(z)
        if l < 3:
            a = np.where(z > 0, z, FC_SLOPE * z)
            acts.append(_bf16_array(a) if bf16 else a)
    d = (dW / st[4]).reshape(9, n * n).T  # dLoss/dout, [P, 9]
    grads = [None] * 4
    for l in range(3, -1, -1):
        grads[l] = d.T @ acts[l]
        if l > 0:
            da = d @ Ws[l]
            d = da * np.where(zs[l - 1] > 0, 1.0, FC_SLOPE)
    return np.concatenate([g.ravel() for g in grads])


def fc_loss_and_grad(st, params, z, omega: float = 2.0 / 3.0, bf16: bool = False, cycles: int = 1):
    """The two-grid objective (eq. twogrid) as a function of the FC network's parameters."""
    W = fc_forward(st, params, omega, bf16)
    loss, dW = twogrid_loss(st, W, z, want_grad=True, cycles=cycles)
    return loss, fc_backward(st, params, dW, omega, bf16)
