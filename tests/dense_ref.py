"""Independent dense-matrix constructions used to pin the oracle.

These build the operators from a different formulation than the oracle's stencil
loops (Kronecker products of 1-D matrices, row-scaled shift matrices, recursive
dense Galerkin products) so that an index, sign or transpose slip in the oracle
shows up as a mismatch.
"""
from __future__ import annotations

import numpy as np


def shift(n: int, d: int) -> np.ndarray:
    """n x n matrix with ones at (i, i+d)."""
    return np.eye(n, k=d)


def field_matrix(st: np.ndarray) -> np.ndarray:
    """A = sum_k diag(st_k) (S_di kron S_dj): row p couples to p + (di, dj) with st_k[p]."""
    n = st.shape[1]
    A = np.zeros((n * n, n * n))
    for k in range(9):
        di, dj = k // 3 - 1, k % 3 - 1
        A += np.diag(st[k].ravel()) @ np.kron(shift(n, di), shift(n, dj))
    return A


def const_matrix(s: np.ndarray, n: int) -> np.ndarray:
    """Constant stencil: A = sum_k s_k (S_di kron S_dj)."""
    s = np.asarray(s).reshape(9)
    A = np.zeros((n * n, n * n))
    for k in range(9):
        di, dj = k // 3 - 1, k % 3 - 1
        A += s[k] * np.kron(shift(n, di), shift(n, dj))
    return A


def interp1d(n: int) -> np.ndarray:
    """1-D linear interpolation, coarse point I at fine 2I+1."""
    nc = (n - 1) // 2
    P = np.zeros((n, nc))
    for I in range(nc):
        P[2 * I + 1, I] = 1.0
        P[2 * I, I] = 0.5
        P[2 * I + 2, I] = 0.5
    return P


def prolongation(n: int) -> np.ndarray:
    P1 = interp1d(n)
    return np.kron(P1, P1)


def kernels_matrix(W: np.ndarray) -> np.ndarray:
    """H[p, p + d_k] = W_k[p]: same construction as field_matrix."""
    return field_matrix(W)


def jacobi_matrix(Al: np.ndarray, omega: float = 2.0 / 3.0) -> np.ndarray:
    return omega * np.diag(1.0 / np.diag(Al))


def vcycle_matrix(A: np.ndarray, ns: list[int], smoother=None, nu1: int = 1, nu2: int = 1, rscale: float = 1.0,
                  mixed: bool = False) -> np.ndarray:
    """Error propagation of the recursive V-cycle with Galerkin coarse operators.

    E_l = S_l^nu2 (I - P_l (I - E_{l+1}) A_{l+1}^{-1} R_l A_l) S_l^nu1, E_last = 0,
    S_l = I - H_l A_l with H_l = smoother(l, A_l) (default weighted Jacobi), restriction
    R_l = rscale P_l^T and A_{l+1} = R_l A_l P_l (mixed: P_l^T A_l P_l whatever rscale).
    """
    smoother = smoother or (lambda l, Al: jacobi_matrix(Al))

    def rec(l: int, Al: np.ndarray) -> np.ndarray:
        n = ns[l]
        I = np.eye(n * n)
        if l == len(ns) - 1:
            return np.zeros_like(Al)
        P = prolongation(n)
        R = rscale * P.T
        Ac = (P.T if mixed else R) @ Al @ P
        Ec = rec(l + 1, Ac)
        S = I - smoother(l, Al) @ Al
        C = I - P @ (np.eye(Ac.shape[0]) - Ec) @ np.linalg.solve(Ac, R @ Al)
        return np.linalg.matrix_power(S, nu2) @ C @ np.linalg.matrix_power(S, nu1)

    return rec(0, A)
