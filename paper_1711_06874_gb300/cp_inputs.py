"""Seeded canonical (CP) inputs of the canonical-to-Tucker route (Sec. 3.4).

A CP tensor A = C x_1 U1 x_2 U2 x_3 U3 (Eq. Can_Contr, Sec. 3.1) is given by its weights
c (length R) and side matrices U_l (n_l x R, unit columns).  This module only
produces such inputs; it holds none of the canonical-to-Tucker arithmetic.

newton_sinc_cp: the paper's example of a CP input, the collocation of the
Newton kernel 1/|x| through the sinc quadrature of its Gaussian integral
(Eq. laplace, Eq. hM, Eq. sinc_Newt).  With a(t) = 1/sqrt(pi) on the whole
real line, 1/p = int a(t) exp(-t^2 p^2) dt, the quadrature nodes are
t_k = k h_M, weights a_k = a(t_k) h_M, k = -M..M, h_M = C_0 log(M) / M, and
each term is separable: exp(-t_k^2 |x|^2) = prod_l exp(-t_k^2 x_l^2).  The
grid points are those of Sec. 3.7 (cell-centred by default).
"""
from __future__ import annotations

import math

import numpy as np

CELL, VERTEX = 0, 1


def grid_points(n: int, b: float = 1.0, kind: int = CELL) -> np.ndarray:
    i = np.arange(n, dtype=np.float64)
    if kind == VERTEX:
        return -b + i * (2.0 * b / (n - 1))
    return -b + (i + 0.5) * (2.0 * b / n)


def newton_sinc_cp(n, M: int, c0: float = 3.0, b=1.0, kind: int = CELL):
    """(c, [U1, U2, U3]) of the R = 2M + 1 term sinc expansion of 1/|x|
    collocated on the n1 x n2 x n3 grid over [-b, b]^3; unit columns, the
    norms moved into c."""
    if M < 2:
        raise ValueError("M >= 2 (h_M = C_0 log(M) / M)")
    n = [int(v) for v in (n if np.ndim(n) else (n, n, n))]
    bs = [float(v) for v in (b if np.ndim(b) else (b, b, b))]
    h = c0 * math.log(M) / M
    k = np.arange(-M, M + 1, dtype=np.float64)
    t = k * h
    a = np.full(t.shape, h / math.sqrt(math.pi))
    c = a.copy()
    U = []
    for l in range(3):
        x = grid_points(n[l], bs[l], kind)
        G = np.exp(-np.outer(x * x, t * t))  # n_l x R
        nrm = np.linalg.norm(G, axis=0)
        U.append(G / nrm)
        c = c * nrm
    return c, U


def random_cp(seed: int, n, R: int, col_rank=None):
    """(c, [U1, U2, U3]) with standard normal entries and weights, unit
    columns; with col_rank (3 ints) each side matrix has exactly that column
    rank (its columns drawn from a random subspace of that dimension)."""
    rng = np.random.default_rng(seed)
    c = rng.standard_normal(R)
    U = []
    for l in range(3):
        if col_rank is None:
            A = rng.standard_normal((n[l], R))
        else:
            A = rng.standard_normal((n[l], col_rank[l])) @ rng.standard_normal((col_rank[l], R))
        U.append(A / np.linalg.norm(A, axis=0))
    return c, U
