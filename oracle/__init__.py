"""Python access to the FP64 CPU oracle (``tucker_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the independent reference for the
Tucker/HOSVD of covariance tensors in arXiv:1711.06874.  Only the test suite,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg use it; the
CUDA library never imports, links or calls anything here.

Parity status of each routine (what pins it) is listed in the C source.
The multigrid Tucker and the canonical-to-Tucker routines at the end of this
file are written in Python over those routines and LAPACK's SVD (numpy);
their pins are in the test suite (test_oracle_pins.py).  The
value of the Tucker tensor at the origin compared with the printed table of
Sec. 4 (Table zero_points) is a sanity check only: the paper does not state
the box size or whether ALS followed the HOSVD, so that comparison is parity
unpinned.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tucker_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MATERN, SLATER_P, GAUSSIAN, MATERN_SD = 0, 1, 2, 3
CELL, VERTEX = 0, 1
RANK_CAPPED, EPS_UNREACHABLE = 1, 2


class Kernel(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("nu", ctypes.c_double),
        ("ell", ctypes.c_double * 3),
        ("sigma2", ctypes.c_double),
        ("p", ctypes.c_double),
    ]


class Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("b", ctypes.c_double * 3), ("kind", ctypes.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(os.path.join(_HERE, "tucker_oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        kp, gp = ctypes.POINTER(Kernel), ctypes.POINTER(Grid)
        sig = {
            "or_bessel_k_scaled": (d, [d, d]),
            "or_bessel_k": (d, [d, d]),
            "or_matern_z": (d, [d, d, d]),
            "or_kernel_value": (d, [kp, p]),
            "or_grid_axis": (None, [i, i, d, p]),
            "or_tensor": (None, [kp, gp, p]),
            "or_unfold": (None, [p, p, i, p]),
            "or_gram": (None, [p, p, i, p]),
            "or_norm2": (d, [p, ctypes.c_longlong]),
            "or_sym_eig": (i, [i, p, p, p]),
            "or_unfolding_svd": (i, [p, p, i, p, p]),
            "or_rank": (i, [p, i, d, d, i, p]),
            "or_core": (None, [p, p, p, i, p, i, p, i, p, p]),
            "or_reconstruct": (None, [p, p, p, i, p, i, p, i, p, p]),
            "or_tucker_point": (d, [p, p, p, i, p, i, p, i, p]),
            "or_rel_error": (d, [p, p, ctypes.c_longlong]),
            "or_hosvd": (i, [kp, gp, d, p, p, p, p, p, p, p, p, p, p, p, p]),
            "or_ttm": (None, [p, p, i, p, i, i, p]),
            "or_hooi": (i, [p, p, p, p, p, p, i, p, p]),
            "or_num_threads": (i, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def make_kernel(kind=MATERN, nu=0.5, ell=1.0, sigma2=1.0, p=1.0) -> Kernel:
    ell3 = [float(ell)] * 3 if np.isscalar(ell) else [float(v) for v in ell]
    return Kernel(int(kind), float(nu), (ctypes.c_double * 3)(*ell3), float(sigma2), float(p))


def make_grid(n, b=1.0, kind=CELL) -> Grid:
    n3 = [int(n)] * 3 if np.isscalar(n) else [int(v) for v in n]
    b3 = [float(b)] * 3 if np.isscalar(b) else [float(v) for v in b]
    return Grid((ctypes.c_int * 3)(*n3), (ctypes.c_double * 3)(*b3), int(kind))


def num_threads() -> int:
    return _load().or_num_threads()


def bessel_k(nu: float, z: float) -> float:
    return _load().or_bessel_k(float(nu), float(z))


def bessel_k_scaled(nu: float, z: float) -> float:
    return _load().or_bessel_k_scaled(float(nu), float(z))


def matern_z(nu: float, sigma2: float, z: float) -> float:
    return _load().or_matern_z(float(nu), float(sigma2), float(z))


def kernel_value(kernel: Kernel, x) -> float:
    x = _f64(x)
    return _load().or_kernel_value(ctypes.byref(kernel), _ptr(x))


def grid_axis(kind: int, n: int, b: float) -> np.ndarray:
    x = np.empty(n, np.float64)
    _load().or_grid_axis(int(kind), int(n), float(b), _ptr(x))
    return x


def tensor(kernel: Kernel, grid: Grid) -> np.ndarray:
    n = tuple(grid.n)
    F = np.empty(n, np.float64)
    _load().or_tensor(ctypes.byref(kernel), ctypes.byref(grid), _ptr(F))
    return F


def unfold(F: np.ndarray, mode: int) -> np.ndarray:
    F = _f64(F)
    n = _i32(F.shape)
    A = np.empty((F.shape[mode], F.size // F.shape[mode]), np.float64)
    _load().or_unfold(_ptr(F), _ptr(n), int(mode), _ptr(A))
    return A


def gram(F: np.ndarray, mode: int) -> np.ndarray:
    F = _f64(F)
    n = _i32(F.shape)
    m = F.shape[mode]
    G = np.empty((m, m), np.float64)
    _load().or_gram(_ptr(F), _ptr(n), int(mode), _ptr(G))
    return G


def norm2(X: np.ndarray) -> float:
    X = _f64(X)
    return _load().or_norm2(_ptr(X), X.size)


def sym_eig(G: np.ndarray):
    """Returns (lam descending, V with eigenvectors as columns, sweeps)."""
    G = _f64(G)
    n = G.shape[0]
    lam = np.empty(n, np.float64)
    V = np.empty((n, n), np.float64)
    sweeps = _load().or_sym_eig(n, _ptr(G), _ptr(lam), _ptr(V))
    return lam, V, sweeps


def unfolding_svd(F: np.ndarray, mode: int):
    F = _f64(F)
    n = _i32(F.shape)
    m = F.shape[mode]
    s = np.empty(m, np.float64)
    U = np.empty((m, m), np.float64)
    _load().or_unfolding_svd(_ptr(F), _ptr(n), int(mode), _ptr(s), _ptr(U))
    return s, U


def rank(lam: np.ndarray, normF2: float, eps: float, rmax: int):
    lam = _f64(lam)
    flags = np.zeros(1, np.int32)
    r = _load().or_rank(_ptr(lam), lam.size, float(normF2), float(eps), int(rmax), _ptr(flags))
    return r, int(flags[0])


def core(F: np.ndarray, U, r) -> np.ndarray:
    F = _f64(F)
    n = _i32(F.shape)
    U = [_f64(u) for u in U]
    r = _i32(r)
    B = np.empty(tuple(int(v) for v in r), np.float64)
    _load().or_core(_ptr(F), _ptr(n), _ptr(U[0]), U[0].shape[1], _ptr(U[1]), U[1].shape[1],
                    _ptr(U[2]), U[2].shape[1], _ptr(r), _ptr(B))
    return B


def reconstruct(B: np.ndarray, U, n) -> np.ndarray:
    B = _f64(B)
    r = _i32(B.shape)
    U = [_f64(u) for u in U]
    n = _i32(n)
    X = np.empty(tuple(int(v) for v in n), np.float64)
    _load().or_reconstruct(_ptr(B), _ptr(r), _ptr(U[0]), U[0].shape[1], _ptr(U[1]), U[1].shape[1],
                           _ptr(U[2]), U[2].shape[1], _ptr(n), _ptr(X))
    return X


def tucker_point(B: np.ndarray, U, idx) -> float:
    B = _f64(B)
    r = _i32(B.shape)
    U = [_f64(u) for u in U]
    idx = _i32(idx)
    return _load().or_tucker_point(_ptr(B), _ptr(r), _ptr(U[0]), U[0].shape[1], _ptr(U[1]),
                                   U[1].shape[1], _ptr(U[2]), U[2].shape[1], _ptr(idx))


def rel_error(F: np.ndarray, X: np.ndarray) -> float:
    F = _f64(F)
    X = _f64(X)
    return _load().or_rel_error(_ptr(F), _ptr(X), F.size)


def ttm(X: np.ndarray, mode: int, U: np.ndarray) -> np.ndarray:
    """Y = X x_mode U^T for U of shape (X.shape[mode], r)."""
    X = _f64(X)
    U = _f64(U)
    d = _i32(X.shape)
    shape = list(X.shape)
    shape[mode] = U.shape[1]
    Y = np.empty(shape, np.float64)
    _load().or_ttm(_ptr(X), _ptr(d), int(mode), _ptr(U), U.shape[1], U.shape[1], _ptr(Y))
    return Y


def hooi(F: np.ndarray, U, sweeps: int):
    """Tucker-ALS (Sec. 3.2) from the starting factors U (n_k x r_k): returns
    (factors, core, core_norm2 after each mode update)."""
    F = _f64(F)
    n = _i32(F.shape)
    U = [_f64(u).copy() for u in U]
    r = _i32([u.shape[1] for u in U])
    B = np.empty(tuple(int(v) for v in r), np.float64)
    hist = np.empty(max(3 * sweeps, 1), np.float64)
    rc = _load().or_hooi(_ptr(F), _ptr(n), _ptr(U[0]), _ptr(U[1]), _ptr(U[2]), _ptr(r), int(sweeps), _ptr(B),
                         _ptr(hist))
    if rc != 0:
        raise MemoryError("oracle hooi failed")
    return U, B, hist[: 3 * sweeps]


def coarser_grid(grid: Grid) -> Grid:
    """The next coarser grid of the dyadic hierarchy (Sec. 3.2, multigrid
    Tucker): the same box with half the cells per axis (cell-centred n -> n/2,
    vertex n -> (n - 1)/2 + 1)."""
    n = [int(v) for v in grid.n]
    if grid.kind == VERTEX:
        if any(v < 3 or (v - 1) % 2 for v in n):
            raise ValueError("vertex grid: n - 1 must be even and n >= 3")
        nc = [(v - 1) // 2 + 1 for v in n]
    else:
        if any(v < 2 or v % 2 for v in n):
            raise ValueError("cell-centred grid: n must be even")
        nc = [v // 2 for v in n]
    return make_grid(nc, b=[float(v) for v in grid.b], kind=int(grid.kind))


def interp_factor(U: np.ndarray, xc: np.ndarray, xf: np.ndarray) -> np.ndarray:
    """Each column of U (given at the coarse points xc) at the fine points xf,
    linearly between the two coarse points around x (continued linearly
    beyond the outermost ones)."""
    U = _f64(U)
    nc = len(xc)
    out = np.empty((len(xf), U.shape[1]), np.float64)
    for i, x in enumerate(xf):
        p = (x - xc[0]) / (xc[1] - xc[0])
        j = min(max(int(math.floor(p)), 0), nc - 2)
        t = p - j
        out[i] = (1.0 - t) * U[j] + t * U[j + 1]
    return out


def multigrid(kernel: Kernel, grid: Grid, eps: float, levels: int, sweeps: int, rmax=None, rfix=None) -> dict:
    """Multigrid Tucker (Sec. 3.2): the HOSVD on the coarsest of levels + 1
    dyadically refined grids only; on each finer grid the factors from the
    grid below, interpolated and orthonormalised, start `sweeps` Tucker-ALS
    sweeps on that grid's tensor.  The ranks are the coarse HOSVD's."""
    grids = [grid]
    for _ in range(levels):
        grids.insert(0, coarser_grid(grids[0]))
    coarse = hosvd(kernel, grids[0], eps, rmax=rmax, rfix=rfix)
    U = coarse["U"]
    for lv, g in enumerate(grids):
        if lv > 0:
            prev = grids[lv - 1]
            U = [np.linalg.qr(interp_factor(U[a], grid_axis(prev.kind, prev.n[a], prev.b[a]),
                                            grid_axis(g.kind, g.n[a], g.b[a])))[0] for a in range(3)]
        F = tensor(kernel, g)
        U, B, hist = hooi(F, U, sweeps)
    X = reconstruct(B, U, list(grid.n))
    return {"ranks": coarse["ranks"], "U": U, "core": B, "core_norm2_hist": hist, "rel_error": rel_error(F, X),
            "normF2": norm2(F), "coarse": coarse}


def hosvd(kernel: Kernel, grid: Grid, eps: float, rmax=None, rfix=None) -> dict:
    """Full HOSVD of the sampled covariance (Sec. 3.2) with the eps rank rule."""
    n = [int(v) for v in grid.n]
    rmax = _i32(n if rmax is None else ([rmax] * 3 if np.isscalar(rmax) else rmax))
    rfix = _i32([0, 0, 0] if rfix is None else ([rfix] * 3 if np.isscalar(rfix) else rfix))
    ranks = np.zeros(3, np.int32)
    flags = np.zeros(3, np.int32)
    U = [np.empty((m, m), np.float64) for m in n]
    lam = [np.empty(m, np.float64) for m in n]
    B = np.empty(n[0] * n[1] * n[2], np.float64)
    out = np.zeros(3, np.float64)
    rc = _load().or_hosvd(ctypes.byref(kernel), ctypes.byref(grid), float(eps), _ptr(rmax),
                          _ptr(rfix), _ptr(ranks), _ptr(flags), _ptr(U[0]), _ptr(U[1]),
                          _ptr(U[2]), _ptr(lam[0]), _ptr(lam[1]), _ptr(lam[2]), _ptr(B), _ptr(out))
    if rc != 0:
        raise MemoryError("oracle hosvd failed")
    r = [int(v) for v in ranks]
    return {
        "ranks": r,
        "flags": [int(v) for v in flags],
        "U": [U[m][:, : r[m]].copy() for m in range(3)],
        "U_all": U,
        "lam": lam,
        "core": B[: r[0] * r[1] * r[2]].reshape(r).copy(),
        "normF2": float(out[0]),
        "rel_error": float(out[1]),
        "core_norm2": float(out[2]),
    }


# ---------------------------------------------------------------------------
# Canonical-to-Tucker (C2T) of Sec. 3.4: the Tucker approximation of a tensor
# given in the canonical format A = C x_1 U1 x_2 U2 x_3 U3, C = diag(c)
# (Eq. Can_Contr, Sec. 3.1), without forming or unfolding A.  The initial
# guess is the reduced HOSVD (RHOSVD): the leading left singular vectors of
# each side matrix U_l; Tucker-ALS sweeps follow, each single-hole unfolding
# taken in the canonical format.  The SVDs are LAPACK's (numpy).
# ---------------------------------------------------------------------------


def _canonical_signs(Z: np.ndarray) -> np.ndarray:
    """Each column's entry of largest magnitude among the first ceil(n/2)
    made positive (the lowest index on a tie), as for the HOSVD factors."""
    Z = Z.copy()
    h = (Z.shape[0] + 1) // 2
    for j in range(Z.shape[1]):
        i = int(np.argmax(np.abs(Z[:h, j])))
        if Z[i, j] < 0:
            Z[:, j] = -Z[:, j]
    return Z


def cp_full(c, U) -> np.ndarray:
    """The full tensor a(i1, i2, i3) = sum_k c_k U1[i1, k] U2[i2, k] U3[i3, k]."""
    c = _f64(c)
    out = np.zeros((U[0].shape[0], U[1].shape[0], U[2].shape[0]), np.float64)
    for k in range(c.size):
        out += c[k] * np.multiply.outer(np.multiply.outer(U[0][:, k], U[1][:, k]), U[2][:, k])
    return out


def cp_norm2(c, U) -> float:
    """|A|_F^2 = sum_{k, k'} c_k c_k' prod_l <u_k^(l), u_k'^(l)>."""
    c = _f64(c)
    G = np.outer(c, c)
    for l in range(3):
        G = G * (U[l].T @ U[l])
    return float(G.sum())


def cp_core(c, W) -> np.ndarray:
    """Core of the projection: B = sum_k c_k W1[:, k] o W2[:, k] o W3[:, k],
    with W_l = Z_l^T U_l (r_l x R)."""
    return cp_full(c, W)


def rhosvd(c, U, eps: float, rmax=None, rfix=None) -> dict:
    """Reduced HOSVD of the canonical tensor (c, U): Z_l = leading left
    singular vectors of U_l (unit columns).  Rank rule: r_l is the smallest r
    whose discarded singular values satisfy sqrt(sum_{k>r} s_k^2) <=
    eps |A| / (3 |c|), so that the RHOSVD bound |A - A_r| <= |c| sum_l
    sqrt(sum_{k>r_l} s_{l,k}^2) guarantees E <= eps; capped at rmax, replaced
    by rfix where that is > 0.  Core B = A x_1 Z1^T x_2 Z2^T x_3 Z3^T,
    formed in the canonical format."""
    c = _f64(c)
    U = [_f64(u) for u in U]
    normA2 = cp_norm2(c, U)
    cn = float(np.linalg.norm(c))
    tol = eps * math.sqrt(max(normA2, 0.0)) / (3.0 * cn) if cn > 0 else 0.0
    Z, W, sv, ranks, delta = [], [], [], [], []
    for l in range(3):
        Ul, s, _ = np.linalg.svd(U[l], full_matrices=False)
        tail = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1])  # tail[r] = sqrt(sum_{k >= r} s_k^2)
        r = s.size
        for q in range(1, s.size + 1):
            if q == s.size or tail[q] <= tol:
                r = q
                break
        if rmax is not None:
            r = min(r, int(rmax[l] if np.ndim(rmax) else rmax))
        if rfix is not None and int(rfix[l]) > 0:
            r = min(int(rfix[l]), s.size)
        Zl = _canonical_signs(Ul[:, :r])
        Z.append(Zl)
        W.append(Zl.T @ U[l])
        sv.append(s)
        ranks.append(r)
        delta.append(float(tail[r]) if r < s.size else 0.0)
    return {"ranks": ranks, "U": Z, "W": W, "sv": sv, "core": cp_core(c, W), "normA2": normA2,
            "bound": cn * sum(delta)}


def c2t(c, U, eps: float, sweeps: int, rmax=None, rfix=None) -> dict:
    """Canonical-to-Tucker (Sec. 3.4): the RHOSVD as the initial guess, then
    `sweeps` Tucker-ALS sweeps over modes 1, 2, 3 (each update using the
    factors already updated in the sweep).  The single-hole tensor of mode l,
    A x_m Z_m^T x_q Z_q^T (m < q the other modes), has the mode-l unfolding
    M[i, a r_q + b] = sum_k U_l[i, k] c_k W_m[a, k] W_q[b, k]; Z_l becomes its
    r_l leading left singular vectors.  Returns the factors, the core and
    |B|^2 after each mode update (the sum of the kept squared singular
    values)."""
    c = _f64(c)
    U = [_f64(u) for u in U]
    init = rhosvd(c, U, eps, rmax=rmax, rfix=rfix)
    r = init["ranks"]
    for l in range(3):
        if r[l] > r[(l + 1) % 3] * r[(l + 2) % 3]:
            raise ValueError("the RHOSVD ranks are not a multilinear rank (r_l > r_m r_q)")
    Z = [z.copy() for z in init["U"]]
    W = [w.copy() for w in init["W"]]
    hist = []
    for _ in range(sweeps):
        for l in range(3):
            m, q = [a for a in range(3) if a != l]
            KR = (W[m][:, None, :] * W[q][None, :, :]).reshape(r[m] * r[q], c.size)  # Khatri-Rao, row a r_q + b
            M = (U[l] * c[None, :]) @ KR.T
            Ul, s, _ = np.linalg.svd(M, full_matrices=False)
            Z[l] = _canonical_signs(Ul[:, : r[l]])
            W[l] = Z[l].T @ U[l]
            hist.append(float((s[: r[l]] ** 2).sum()))
    return {"ranks": r, "U": Z, "core": cp_core(c, W), "core_norm2_hist": np.array(hist), "rhosvd": init}
