"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test ties one oracle routine to something other than itself: a closed
form, an identity, a library routine on a special case, brute force on tiny
inputs, or a value printed in the paper.  The mutation tests at the end plant
plausible mistakes (on the CPU, in the oracle's inputs and outputs) and show
that the pins catch them.
"""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# K_nu and the Matern function (Sec. 2.2, Eq. (Matern))
# --------------------------------------------------------------------------
ZS = [1e-4, 3e-3, 0.052, 0.09, 0.5, 1.0, 1.9, 2.0, 2.1, 5.7, 13.4, 38.7, 77.3, 250.0]


@pytest.mark.parametrize("z", ZS)
def test_bessel_half_integer_closed_forms(orc, z):
    # K_{1/2}, K_{3/2}, K_{5/2} are elementary (K_{n+1/2} closed forms).
    base = math.sqrt(math.pi / (2 * z))
    want = {
        0.5: base,
        1.5: base * (1 + 1 / z),
        2.5: base * (1 + 3 / z + 3 / z ** 2),
    }
    for nu, w in want.items():
        got = orc.bessel_k_scaled(nu, z)  # K * e^z
        assert abs(got - w) <= 2e-15 * abs(w), (nu, z, got, w)


@pytest.mark.parametrize("nu", [0.3, 0.8, 1.2, 2.3, 3.7])
def test_bessel_order_recurrence(orc, nu):
    # K_{nu+1}(z) - K_{nu-1}(z) = (2 nu / z) K_nu(z)
    for z in ZS[:-1]:
        kp = orc.bessel_k_scaled(nu + 1, z)
        km = orc.bessel_k_scaled(nu - 1, z)
        k0 = orc.bessel_k_scaled(nu, z)
        assert abs((kp - km) - 2 * nu / z * k0) <= 5e-15 * kp, (nu, z)


def test_bessel_matches_scipy(orc):
    sp = pytest.importorskip("scipy.special")
    # scipy's kv itself carries errors up to ~5e-14 near z = 2
    for nu in [0.3, 0.5, 1.2, 2.5]:
        for z in ZS[:-1]:
            a, b = orc.bessel_k(nu, z), float(sp.kv(nu, z))
            assert abs(a - b) <= 2e-13 * abs(b), (nu, z, a, b)


def test_bessel_matches_mpmath(orc):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for nu in [0.3, 1.2, 2.5, 0.75]:
        for z in [1e-3, 0.5, 2.0, 13.4, 77.3]:
            ex = float(mp.besselk(nu, z) * mp.e ** z)
            got = orc.bessel_k_scaled(nu, z)
            assert abs(got - ex) <= 2e-15 * ex, (nu, z, got, ex)


@pytest.mark.parametrize("z", [1e-6, 0.09, 0.7, 3.0, 13.4, 38.7])
def test_matern_closed_forms(orc, z):
    # nu = 1/2 is the exponential model (Sec. 2.2); 3/2 and 5/2 follow from
    # the elementary K_{n+1/2}.  Here z = sqrt(2 nu) r / ell.
    s2 = 1.7
    want = {
        0.5: s2 * math.exp(-z),
        1.5: s2 * (1 + z) * math.exp(-z),
        2.5: s2 * (1 + z + z * z / 3) * math.exp(-z),
    }
    for nu, w in want.items():
        got = orc.matern_z(nu, s2, z)
        # z^nu e^-z is formed as exp(nu log z - z): rounding of the exponent
        # costs about |nu log z| + z ulps
        assert abs(got - w) <= (4 + abs(nu * math.log(z)) + z) * 2.3e-16 * w, (nu, z, got, w)


def test_matern_small_r_limit_and_origin(orc):
    assert orc.matern_z(1.2, 2.5, 0.0) == 2.5
    # C(z) = sigma2 (1 - O(z^2)) for nu > 1
    assert abs(orc.matern_z(1.2, 2.5, 1e-6) / 2.5 - 1) < 1e-10
    assert abs(orc.matern_z(0.3, 1.0, 1e-12) - 1) < 1e-6


def test_matern_gaussian_limit(orc):
    # nu -> infinity gives the Gaussian model (Sec. 2.2): C -> exp(-r^2 / (2 ell^2))
    for rho in [0.5, 1.0, 1.5]:
        nu = 200.0
        got = orc.matern_z(nu, 1.0, math.sqrt(2 * nu) * rho)
        assert abs(got - math.exp(-rho * rho / 2)) < 3e-3 * math.exp(-rho * rho / 2) + 1e-3


def test_kernel_value_anisotropic(orc):
    # r_A^2 = sum x_a^2 / ell_a^2 (Sec. 2.2, diagonal A)
    k = orc.make_kernel(orc.MATERN, nu=1.5, ell=[0.3, 0.5, 0.7], sigma2=1.3)
    x = [0.1, -0.2, 0.35]
    ra = math.sqrt(sum((xi / li) ** 2 for xi, li in zip(x, [0.3, 0.5, 0.7])))
    z = math.sqrt(3.0) * ra
    assert abs(orc.kernel_value(k, x) - 1.3 * (1 + z) * math.exp(-z)) < 1e-15
    ks = orc.make_kernel(orc.SLATER_P, ell=1.0, p=0.2)
    assert abs(orc.kernel_value(ks, [0.3, 0.4, 0.0]) - math.exp(-(0.5 ** 0.2))) < 1e-15
    kg = orc.make_kernel(orc.GAUSSIAN, ell=0.5, sigma2=2.0)
    assert abs(orc.kernel_value(kg, [0.1, 0.2, 0.3]) - 2.0 * math.exp(-0.14 / 0.25)) < 1e-15


# --------------------------------------------------------------------------
# Grid and collocation tensor (Sec. 3.7, Eq. (grid_points))
# --------------------------------------------------------------------------
def test_grid_axes(orc):
    np.testing.assert_array_equal(orc.grid_axis(orc.CELL, 4, 1.0), [-0.75, -0.25, 0.25, 0.75])
    np.testing.assert_array_equal(orc.grid_axis(orc.VERTEX, 5, 2.0), [-2.0, -1.0, 0.0, 1.0, 2.0])
    x = orc.grid_axis(orc.CELL, 64, 1.0)
    np.testing.assert_allclose(x, -1 + (np.arange(64) + 0.5) * 2 / 64, rtol=0, atol=1e-16)


def test_tensor_entries_and_symmetry(orc):
    k = orc.make_kernel(orc.MATERN, nu=1.2, ell=[0.2, 0.3, 0.4])
    g = orc.make_grid([5, 6, 7], b=[1.0, 0.8, 1.2])
    F = orc.tensor(k, g)
    xs = [orc.grid_axis(orc.CELL, n, b) for n, b in zip([5, 6, 7], [1.0, 0.8, 1.2])]
    for (i, j, l) in [(0, 0, 0), (2, 3, 4), (4, 5, 6), (1, 2, 0)]:
        assert F[i, j, l] == orc.kernel_value(k, [xs[0][i], xs[1][j], xs[2][l]])
    # even function on a symmetric grid (mirrored coordinates agree to rounding)
    np.testing.assert_allclose(F, F[::-1, :, :], rtol=1e-14)
    np.testing.assert_allclose(F, F[:, ::-1, ::-1], rtol=1e-14)


# --------------------------------------------------------------------------
# Unfolding and Gram (Sec. 3.2, Fig. Unfolding)
# --------------------------------------------------------------------------
def test_unfolding_matches_numpy(orc):
    rng = np.random.default_rng(0)
    F = rng.standard_normal((3, 4, 5))
    np.testing.assert_array_equal(orc.unfold(F, 0), F.reshape(3, 20))
    np.testing.assert_array_equal(orc.unfold(F, 1), F.transpose(1, 0, 2).reshape(4, 15))
    np.testing.assert_array_equal(orc.unfold(F, 2), F.transpose(2, 0, 1).reshape(5, 12))


def test_gram_against_matmul_and_trace(orc):
    rng = np.random.default_rng(1)
    F = rng.random((6, 7, 9))
    for m in range(3):
        A = np.moveaxis(F, m, 0).reshape(F.shape[m], -1)
        G = orc.gram(F, m)
        np.testing.assert_allclose(G, A @ A.T, rtol=1e-14)
        assert abs(np.trace(G) - orc.norm2(F)) <= 1e-14 * orc.norm2(F)


def test_gram_isotropy_and_persymmetry(orc):
    k = orc.make_kernel(orc.MATERN, nu=0.8, ell=0.25)
    F = orc.tensor(k, orc.make_grid(12))
    G = [orc.gram(F, m) for m in range(3)]
    np.testing.assert_allclose(G[0], G[1], rtol=1e-15)
    np.testing.assert_allclose(G[0], G[2], rtol=1e-15)
    np.testing.assert_allclose(G[0], G[0][::-1, ::-1], rtol=1e-14)  # mirrored grid points round differently


REFLECT_CASES = [  # (n, ell, grid kind): even/odd axes, anisotropic, both grids
    ((10, 9, 7), (0.3, 0.5, 0.7), 0),
    ((8, 11, 6), (0.4, 0.2, 0.9), 1),
    ((9, 9, 9), (0.25, 0.25, 0.25), 1),
]


def _octant(F):
    """sqrt(w_i w_j w_l) F on the upper octant, w = 1 at an odd axis' centre, else 2."""
    out = F[tuple(slice(m // 2, m) for m in F.shape)].copy()
    for a, m in enumerate(F.shape):
        w = np.full(m - m // 2, 2.0)
        if m % 2:
            w[0] = 1.0
        shp = [1, 1, 1]
        shp[a] = -1
        out *= np.sqrt(w).reshape(shp)
    return out


@pytest.mark.parametrize("case", REFLECT_CASES)
def test_gram_odd_half_vanishes(orc, case):
    """C depends on x_a only through x_a^2 and the grid is symmetric, so rows
    i and n-1-i of every unfolding coincide: G_k J = G_k, and G_k has at most
    ceil(n_k/2) nonzero eigenvalues."""
    n, ell, kind = case
    F = orc.tensor(orc.make_kernel(orc.MATERN, nu=1.3, ell=list(ell)), orc.make_grid(list(n), kind=kind))
    for m in range(3):
        G = orc.gram(F, m)
        np.testing.assert_allclose(G[:, ::-1], G, rtol=0, atol=1e-14 * np.abs(G).max())
        lam, _, _ = orc.sym_eig(G)
        h = (n[m] + 1) // 2
        assert np.abs(lam[h:]).max(initial=0.0) <= 1e-14 * lam[0]


@pytest.mark.parametrize("case", REFLECT_CASES)
def test_octant_gram_has_the_even_spectrum(orc, case):
    """The weighted octant keeps |F| and its Gram has the leading eigenvalues
    of G_k (numpy on the octant against the oracle on the whole tensor)."""
    n, ell, kind = case
    F = orc.tensor(orc.make_kernel(orc.MATERN, nu=0.9, ell=list(ell)), orc.make_grid(list(n), kind=kind))
    Fh = _octant(F)
    assert abs(np.sum(Fh ** 2) - np.sum(F ** 2)) <= 1e-14 * np.sum(F ** 2)
    for m in range(3):
        lam, _, _ = orc.sym_eig(orc.gram(F, m))
        A = np.moveaxis(Fh, m, 0).reshape(Fh.shape[m], -1)
        mu = np.sort(np.linalg.eigvalsh(A @ A.T))[::-1]
        np.testing.assert_allclose(mu, lam[: len(mu)], rtol=0, atol=1e-13 * lam[0])


# --------------------------------------------------------------------------
# Jacobi eigensolver
# --------------------------------------------------------------------------
def test_sym_eig_random(orc):
    rng = np.random.default_rng(2)
    for n in [1, 2, 5, 17, 40]:
        A = rng.standard_normal((n, n))
        A = A + A.T
        lam, V, _ = orc.sym_eig(A)
        ref = np.sort(np.linalg.eigvalsh(A))[::-1]
        np.testing.assert_allclose(lam, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
        np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-14)
        np.testing.assert_allclose(V @ np.diag(lam) @ V.T, A, atol=2e-14 * np.abs(A).max() * n)
        # canonical sign: largest |entry| in the first half of each column is positive
        h = (n + 1) // 2
        for j in range(n):
            i = int(np.argmax(np.abs(V[:h, j])))
            assert V[i, j] > 0


def test_sym_eig_graded_psd(orc):
    # geometric spectrum like the Grams here: eigenvalues resolved to u * lam_1
    rng = np.random.default_rng(3)
    n = 30
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    d = 10.0 ** (-np.arange(n) * 0.7)
    A = (Q * d) @ Q.T
    lam, V, _ = orc.sym_eig(A)
    np.testing.assert_allclose(lam, d, rtol=0, atol=4e-16 * n)
    for j in range(8):  # well separated leading vectors
        assert abs(abs(V[:, j] @ Q[:, j]) - 1) < 1e-12


# --------------------------------------------------------------------------
# HOSVD (Sec. 3.2) against brute force and structural facts
# --------------------------------------------------------------------------
def _principal_sines(U, W):
    # sines of the principal angles: singular values of (I - U U^T) W
    # (1 - cos^2 would lose half the digits)
    return np.linalg.svd(W - U @ (U.T @ W), compute_uv=False)


def test_hosvd_small_matches_numpy_svd_of_unfoldings(orc):
    k = orc.make_kernel(orc.MATERN, nu=1.2, ell=[0.4, 0.6, 0.9])
    g = orc.make_grid([6, 7, 8])
    F = orc.tensor(k, g)
    res = orc.hosvd(k, g, 0.0, rfix=[6, 7, 8])
    for m in range(3):
        A = np.moveaxis(F, m, 0).reshape(F.shape[m], -1)
        Us, s, _ = np.linalg.svd(A, full_matrices=False)
        lam = res["lam"][m]
        np.testing.assert_allclose(lam, s ** 2, rtol=0, atol=2e-14 * s[0] ** 2)
        # leading well-separated singular vectors agree as subspaces
        for j in range(3):
            assert _principal_sines(res["U_all"][m][:, : j + 1], Us[:, : j + 1]).max() < 1e-10


def test_hosvd_second_route_one_sided_jacobi(orc):
    k = orc.make_kernel(orc.MATERN, nu=0.5, ell=0.3)
    F = orc.tensor(k, orc.make_grid(8))
    for m in range(3):
        sig, U = orc.unfolding_svd(F, m)
        lam, V, _ = orc.sym_eig(orc.gram(F, m))
        np.testing.assert_allclose(sig ** 2, lam, rtol=0, atol=1e-14 * lam[0])
        for j in range(4):
            assert abs(abs(U[:, j] @ V[:, j]) - 1) < 1e-12


def test_gaussian_is_rank_one(orc):
    # exp(-|x|^2/ell^2) = prod_a exp(-x_a^2/ell^2): a rank-1 tensor (Sec. 3.1, 4.4)
    k = orc.make_kernel(orc.GAUSSIAN, ell=0.4)
    res = orc.hosvd(k, orc.make_grid(16), 1e-6)
    assert res["ranks"] == [1, 1, 1]
    assert res["rel_error"] <= 1e-14


def test_full_rank_is_exact(orc):
    k = orc.make_kernel(orc.MATERN, nu=0.5, ell=0.3)
    res = orc.hosvd(k, orc.make_grid([9, 10, 11]), 0.0, rfix=[9, 10, 11])
    assert res["rel_error"] <= 1e-13
    assert abs(res["core_norm2"] - res["normF2"]) <= 1e-14 * res["normF2"]


@pytest.mark.parametrize("nu,ell,eps", [(0.5, 0.3, 1e-4), (1.2, 0.2, 1e-6), (2.5, 0.1, 1e-6), (0.3, 0.05, 1e-4)])
def test_hosvd_error_bound(orc, nu, ell, eps):
    # |F - X|^2 <= sum_k sum_{i > r_k} lam_i^(k)  (HOSVD bound), and the eps split
    k = orc.make_kernel(orc.MATERN, nu=nu, ell=ell)
    res = orc.hosvd(k, orc.make_grid(20), eps)
    disc = sum(np.clip(res["lam"][m][res["ranks"][m]:], 0, None).sum() for m in range(3))
    e2 = res["rel_error"] ** 2 * res["normF2"]
    assert e2 <= disc * (1 + 1e-9) + 1e-28 * res["normF2"]
    assert res["rel_error"] <= eps
    # orthogonal factors: |F - X|^2 = |F|^2 - |B|^2
    assert abs(e2 - (res["normF2"] - res["core_norm2"])) <= 1e-13 * res["normF2"]


def test_sigma2_scaling_invariance(orc):
    g = orc.make_grid(14)
    a = orc.hosvd(orc.make_kernel(orc.MATERN, nu=1.2, ell=0.2, sigma2=1.0), g, 1e-6)
    b = orc.hosvd(orc.make_kernel(orc.MATERN, nu=1.2, ell=0.2, sigma2=3.5), g, 1e-6)
    assert a["ranks"] == b["ranks"]
    assert abs(a["rel_error"] - b["rel_error"]) <= 1e-12
    for m in range(3):
        assert _principal_sines(a["U"][m][:, :4], b["U"][m][:, :4]).max() < 1e-10
    np.testing.assert_allclose(b["core"][0, 0, 0], 3.5 * a["core"][0, 0, 0], rtol=1e-13)


def test_d2_reduces_to_matrix_svd(orc):
    # For d = 2 the orthogonal Tucker decomposition is the SVD (Sec. 3.1).
    k = orc.make_kernel(orc.MATERN, nu=1.5, ell=[0.3, 0.5, 1.0])
    g = orc.make_grid([9, 7, 1])
    F = orc.tensor(k, g)
    M = F[:, :, 0]
    U, s, Vt = np.linalg.svd(M)
    res = orc.hosvd(k, g, 0.0, rfix=[7, 7, 1])
    B = res["core"][:, :, 0]
    np.testing.assert_allclose(np.abs(np.diag(B)), s, rtol=0, atol=1e-14 * s[0])
    off = B - np.diag(np.diag(B))
    assert np.abs(off).max() <= 1e-13 * s[0]
    for j in range(3):
        assert abs(abs(res["U"][0][:, j] @ U[:, j]) - 1) < 1e-12
        assert abs(abs(res["U"][1][:, j] @ Vt[j]) - 1) < 1e-12


def test_rank_rule_by_hand(orc):
    lam = np.array([1.0, 1e-2, 1e-4, 1e-6, -1e-18])
    nf = lam[:4].sum()
    # thr = eps^2 nf / 3; discarded(r) = sum_{i >= r} lam_i^+ (0-based)
    assert orc.rank(lam, nf, math.sqrt(3 * 2e-6 / nf), 10) == (3, 0)   # 1e-6 <= 2e-6 < 1.01e-4
    assert orc.rank(lam, nf, math.sqrt(3 * 1e-6 / nf), 10)[0] == 3    # boundary is inclusive
    assert orc.rank(lam, nf, math.sqrt(3 * 0.99e-6 / nf), 10)[0] == 4
    assert orc.rank(lam, nf, 1.0, 10)[0] == 1
    r, f = orc.rank(lam, nf, 1e-12, 2)
    assert r == 2 and f & orc.RANK_CAPPED
    assert orc.rank(lam, nf, 1e-9, 10)[1] & orc.EPS_UNREACHABLE


def test_core_and_reconstruct_match_einsum(orc):
    rng = np.random.default_rng(4)
    F = rng.standard_normal((5, 6, 7))
    U = [np.linalg.qr(rng.standard_normal((n, n)))[0][:, :r] for n, r in zip(F.shape, (2, 3, 4))]
    B = orc.core(F, U, [2, 3, 4])
    np.testing.assert_allclose(B, np.einsum("ijk,ia,jb,kc->abc", F, *U), atol=1e-13)
    X = orc.reconstruct(B, U, F.shape)
    np.testing.assert_allclose(X, np.einsum("abc,ia,jb,kc->ijk", B, *U), atol=1e-13)
    assert abs(orc.tucker_point(B, U, [1, 2, 3]) - X[1, 2, 3]) < 1e-13
    assert abs(orc.rel_error(F, X) - np.linalg.norm(F - X) / np.linalg.norm(F)) < 1e-14


# --------------------------------------------------------------------------
# The paper's printed table (Sec. 4, Table zero_points): sanity only
# --------------------------------------------------------------------------
def test_zero_points_table_sanity(orc):
    rows = {}
    with open(os.path.join(GOLDEN, "zero_points.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v = line.split()
                rows[int(v[0])] = [float(t) for t in v[1:]]
    n = 129
    # Reading: box b = 5 (not stated in the paper); HOSVD without ALS.
    k = orc.make_kernel(orc.SLATER_P, ell=1.0, p=1.0)
    g = orc.make_grid(n, b=5.0, kind=orc.VERTEX)
    F = orc.tensor(k, g)
    assert F[n // 2, n // 2, n // 2] == 1.0
    lam, V, _ = orc.sym_eig(orc.gram(F, 0))
    for r in range(1, 10):
        U = [V[:, :r]] * 3
        err = 1 - orc.tucker_point(orc.core(F, U, [r] * 3), U, [n // 2] * 3)
        want = rows[129][r - 1]
        assert want / 1.35 <= err <= want * 1.35, (r, err, want)


# --------------------------------------------------------------------------
# Planted mistakes: each must make a pin fail
# --------------------------------------------------------------------------
def test_planted_transposed_factor_is_caught(orc):
    # a transposed factor breaks the HOSVD bound at truncated rank
    k = orc.make_kernel(orc.MATERN, nu=0.5, ell=[0.3, 0.4, 0.5])
    g = orc.make_grid([6, 7, 8])
    F = orc.tensor(k, g)
    res = orc.hosvd(k, g, 0.0, rfix=[6, 7, 8])
    U, lam = res["U_all"], res["lam"]
    r = [3, 3, 3]
    bound = sum(np.clip(lam[m][r[m]:], 0, None).sum() for m in range(3)) / res["normF2"]
    good = [U[0][:, :3], U[1][:, :3], U[2][:, :3]]
    bad = [U[0][:, :3], U[1][:, :3], U[2].T[:, :3].copy()]
    eg = orc.rel_error(F, orc.reconstruct(orc.core(F, good, r), good, F.shape))
    eb = orc.rel_error(F, orc.reconstruct(orc.core(F, bad, r), bad, F.shape))
    assert eg ** 2 <= bound * (1 + 1e-9)
    assert eb ** 2 > bound * 10


def test_planted_dropped_gram_term_is_caught(orc):
    k = orc.make_kernel(orc.MATERN, nu=1.2, ell=0.3)
    F = orc.tensor(k, orc.make_grid(8))
    G = orc.gram(F, 0)
    Fd = F.copy()
    Fd[:, -1, -1] = 0.0  # one column of the unfolding dropped
    Gd = orc.gram(Fd, 0)
    # trace(G) = |F|^2 catches the dropped column
    assert abs(np.trace(Gd) - orc.norm2(F)) > 1e-10 * orc.norm2(F)
    assert abs(np.trace(G) - orc.norm2(F)) <= 1e-14 * orc.norm2(F)


def test_planted_wrong_sign_in_bessel_is_caught(orc):
    # K_{nu+1} + K_{nu-1} in place of the difference fails the recurrence pin
    nu, z = 1.2, 0.7
    kp, km, k0 = (orc.bessel_k(nu + 1, z), orc.bessel_k(nu - 1, z), orc.bessel_k(nu, z))
    assert abs((kp + km) - 2 * nu / z * k0) > 1e-3 * kp


# ---------------------------------------------------------------------------
# Spectral density of the Matern covariance (Sec. 3.7, Eq. (SD_matern), d = 3)
# ---------------------------------------------------------------------------
def test_spectral_density_closed_values(orc):
    """nu = 1/2 makes the exponent nu + 3/2 = 2: on the 3-point vertex grid of
    [-1, 1] with alpha = 1 the values are 1/(1 + r^2)^2 at r^2 = 0, 1, 2, 3."""
    k = orc.make_kernel(orc.MATERN_SD, nu=0.5, ell=1.0, sigma2=2.0, p=1.0)
    F = orc.tensor(k, orc.make_grid([3, 3, 3], b=[1.0, 1.0, 1.0], kind=1))
    assert F[1, 1, 1] == 2.0
    assert F[2, 1, 1] == 0.5 and F[1, 0, 1] == 0.5
    assert abs(F[2, 2, 1] - 2.0 / 9.0) <= 1e-16
    assert F[0, 2, 0] == 2.0 / 16.0


def test_spectral_density_scaling_law(orc):
    """f_{alpha,nu}(x) = alpha^-(2 nu + 3) f_{1,nu}(x / alpha): the tensor on the
    box b with alpha equals the alpha = 1 tensor on the box b / alpha times
    alpha^-(2 nu + 3), for several nu and alpha (pins the exponent and where
    alpha enters)."""
    for nu, alpha in ((0.4, 0.1), (1.3, 2.0), (2.5, 100.0)):
        b = 1.0
        Fa = orc.tensor(orc.make_kernel(orc.MATERN_SD, nu=nu, ell=1.0, p=alpha),
                        orc.make_grid([9, 10, 11], b=[b, b, b], kind=0))
        F1 = orc.tensor(orc.make_kernel(orc.MATERN_SD, nu=nu, ell=1.0, p=1.0),
                        orc.make_grid([9, 10, 11], b=[b / alpha] * 3, kind=0))
        np.testing.assert_allclose(Fa, F1 * alpha ** (-(2 * nu + 3)), rtol=1e-13, atol=0)


def test_spectral_density_anisotropic_scaling(orc):
    """The anisotropic distance r_A^2 = sum x_a^2 / ell_a^2 of Sec. 2.2: scaling
    axis a of the box by ell_a leaves the tensor of ell = (ell_1, ell_2, ell_3)
    equal to the isotropic ell = 1 tensor."""
    ell = (0.5, 2.0, 3.0)
    Fa = orc.tensor(orc.make_kernel(orc.MATERN_SD, nu=0.7, ell=list(ell), p=0.3),
                    orc.make_grid([7, 8, 9], b=list(ell), kind=0))
    F1 = orc.tensor(orc.make_kernel(orc.MATERN_SD, nu=0.7, ell=1.0, p=0.3),
                    orc.make_grid([7, 8, 9], b=[1.0, 1.0, 1.0], kind=0))
    np.testing.assert_allclose(Fa, F1, rtol=1e-14, atol=0)


# --------------------------------------------------------------------------
# Tucker-ALS (Sec. 3.2, the alternating sweeps after the HOSVD)
# --------------------------------------------------------------------------
def _orthonormal(rng, n, r):
    q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return q


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_ttm_matches_einsum(orc, mode):
    rng = np.random.default_rng(40 + mode)
    X = rng.standard_normal((5, 6, 7))
    U = rng.standard_normal((X.shape[mode], 3))
    spec = {0: "ijk,ia->ajk", 1: "ijk,ja->iak", 2: "ijk,ka->ija"}[mode]
    np.testing.assert_allclose(orc.ttm(X, mode, U), np.einsum(spec, X, U), rtol=0, atol=1e-13)


def test_hooi_matrix_case_reaches_eckart_young(orc):
    """With n3 = 1 the tensor is a matrix A and the sweeps are subspace
    iteration on A: from a random start they reach the Eckart-Young optimum,
    |B|^2 = sum of the r leading sigma_i^2 of A, and U1, U2 span A's leading
    singular subspaces."""
    rng = np.random.default_rng(7)
    n1, n2, r = 9, 11, 3
    s = 2.0 ** -np.arange(n1)
    A = _orthonormal(rng, n1, n1) @ np.diag(s) @ _orthonormal(rng, n2, n1).T
    F = A.reshape(n1, n2, 1)
    U0 = [_orthonormal(rng, n1, r), _orthonormal(rng, n2, r), np.ones((1, 1))]
    U, B, hist = orc.hooi(F, U0, sweeps=40)
    assert abs(hist[-1] - np.sum(s[:r] ** 2)) <= 1e-13 * np.sum(s ** 2)
    assert abs(orc.norm2(B) - np.sum(s[:r] ** 2)) <= 1e-13 * np.sum(s ** 2)
    Us, _, Vt = np.linalg.svd(A)
    np.testing.assert_allclose(U[0] @ U[0].T, Us[:, :r] @ Us[:, :r].T, atol=1e-10)
    np.testing.assert_allclose(U[1] @ U[1].T, Vt[:r].T @ Vt[:r], atol=1e-10)


def test_hooi_recovers_exact_multilinear_rank(orc):
    """F = G x_1 A x_2 B x_3 C has multilinear rank (3, 4, 2): one sweep from a
    random start already spans each range (the single-hole unfoldings have the
    column space of the factor), so X = F to rounding."""
    rng = np.random.default_rng(11)
    n, r = (7, 8, 9), (3, 4, 2)
    G = rng.standard_normal(r)
    Q = [_orthonormal(rng, n[a], r[a]) for a in range(3)]
    F = np.einsum("abc,ia,jb,kc->ijk", G, *Q)
    U0 = [_orthonormal(rng, n[a], r[a]) for a in range(3)]
    U, B, hist = orc.hooi(F, U0, sweeps=1)
    X = orc.reconstruct(B, U, n)
    assert orc.rel_error(F, X) <= 1e-13
    assert abs(hist[-1] - orc.norm2(F)) <= 1e-13 * orc.norm2(F)
    for a in range(3):
        np.testing.assert_allclose(U[a] @ U[a].T, Q[a] @ Q[a].T, atol=1e-12)


def test_hooi_is_monotone_and_orthogonal_on_covariance(orc):
    """From the HOSVD factors of an anisotropic Matern tensor: each update
    maximises |B| over one factor, so the history never decreases and starts
    at or above the HOSVD core norm; X is an orthogonal projection of F, so
    |F|^2 = |B|^2 + |F - X|^2; E does not exceed the HOSVD's."""
    k = orc.make_kernel(orc.MATERN, nu=0.7, ell=[0.3, 0.5, 0.8])
    g = orc.make_grid([14, 16, 18], b=[1.0, 1.0, 1.0])
    F = orc.tensor(k, g)
    ref = orc.hosvd(k, g, 1e-3, rfix=[4, 3, 2])
    U, B, hist = orc.hooi(F, ref["U"], sweeps=4)
    nF2 = ref["normF2"]
    assert hist[0] >= ref["core_norm2"] - 1e-14 * nF2
    assert np.all(np.diff(hist) >= -1e-14 * nF2)
    assert hist[-1] > ref["core_norm2"]
    X = orc.reconstruct(B, U, g.n)
    d2 = orc.norm2(F - X)
    assert abs(nF2 - orc.norm2(B) - d2) <= 1e-12 * nF2
    assert orc.rel_error(F, X) <= ref["rel_error"]
    for a in range(3):
        np.testing.assert_allclose(U[a].T @ U[a], np.eye(U[a].shape[1]), atol=1e-13)


def test_hooi_keeps_the_rank_one_gaussian(orc):
    """The Gaussian exp(-r^2) is a product of three vectors: its HOSVD factors
    at rank (1, 1, 1) are already optimal, so the sweeps leave them and the
    core unchanged and X = F."""
    k = orc.make_kernel(orc.GAUSSIAN, ell=[0.4, 0.6, 0.9])
    g = orc.make_grid([10, 11, 12], b=[1.0, 1.0, 1.0])
    F = orc.tensor(k, g)
    ref = orc.hosvd(k, g, 1e-3, rfix=[1, 1, 1])
    U, B, _ = orc.hooi(F, ref["U"], sweeps=2)
    for a in range(3):
        np.testing.assert_allclose(U[a], ref["U"][a], rtol=0, atol=1e-14)
    assert abs(B.item() - ref["core"].item()) <= 1e-14 * abs(ref["core"].item())
    assert orc.rel_error(F, orc.reconstruct(B, U, g.n)) <= 1e-14


def test_planted_als_ordering_mistake_is_caught(orc):
    """A sweep that keeps the trailing instead of the leading singular vectors
    (a sort-order mistake) fails the exact-rank recovery pin, which the same
    sweep with the leading vectors passes."""
    rng = np.random.default_rng(11)
    n, r = (7, 8, 9), (3, 4, 2)
    G = rng.standard_normal(r)
    Q = [_orthonormal(rng, n[a], r[a]) for a in range(3)]
    F = np.einsum("abc,ia,jb,kc->ijk", G, *Q)
    U0 = [_orthonormal(rng, n[a], r[a]) for a in range(3)]

    def sweep(pick):
        U = [u.copy() for u in U0]
        for k in range(3):
            m1, m2 = [a for a in range(3) if a != k]
            Y = orc.ttm(orc.ttm(F, m1, U[m1]), m2, U[m2])
            _, W = orc.unfolding_svd(Y, k)
            U[k] = pick(W, r[k])
        return orc.rel_error(F, orc.reconstruct(orc.core(F, U, r), U, n))

    assert sweep(lambda W, q: W[:, :q]) <= 1e-13
    assert sweep(lambda W, q: W[:, -q:]) > 1e-3


# --------------------------------------------------------------------------
# Multigrid Tucker (Sec. 3.2: HOSVD on the coarsest grid, interpolated
# subspaces and ALS on the finer ones)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind,nf", [(0, 16), (1, 17)])
def test_interp_factor_reproduces_affine_columns(orc, kind, nf):
    """Linear interpolation (and its linear continuation at the ends) is exact
    on affine functions of x, on both grid kinds."""
    gf = orc.make_grid(nf, b=1.3, kind=kind)
    gc = orc.coarser_grid(gf)
    xc = orc.grid_axis(kind, gc.n[0], 1.3)
    xf = orc.grid_axis(kind, nf, 1.3)
    U = np.stack([np.ones_like(xc), xc, 2.0 - 0.5 * xc], axis=1)
    want = np.stack([np.ones_like(xf), xf, 2.0 - 0.5 * xf], axis=1)
    np.testing.assert_allclose(orc.interp_factor(U, xc, xf), want, rtol=0, atol=1e-14)


def test_planted_interpolation_coordinates_are_caught(orc):
    """Interpolating on the vertex coordinates of a cell-centred grid fails
    the affine pin."""
    xc = orc.grid_axis(orc.CELL, 8, 1.0)
    xf_wrong = orc.grid_axis(orc.VERTEX, 16, 1.0)
    xf = orc.grid_axis(orc.CELL, 16, 1.0)
    got = orc.interp_factor(xc[:, None], xc, xf_wrong)
    assert np.abs(got[:, 0] - xf).max() > 1e-3


def test_multigrid_coarser_grid_sizes(orc):
    g = orc.coarser_grid(orc.make_grid([64, 32, 16]))
    assert list(g.n) == [32, 16, 8]
    g = orc.coarser_grid(orc.make_grid([65, 33, 17], kind=orc.VERTEX))
    assert list(g.n) == [33, 17, 9]
    with pytest.raises(ValueError):
        orc.coarser_grid(orc.make_grid([15, 16, 16]))


def test_multigrid_rank_one_gaussian_is_exact(orc):
    """The Gaussian is separable: from the coarse rank-one factors the fine
    sweeps recover it to rounding."""
    k = orc.make_kernel(orc.GAUSSIAN, ell=[0.5, 0.7, 0.9])
    out = orc.multigrid(k, orc.make_grid([32, 32, 32]), 1e-3, levels=2, sweeps=1, rfix=[1, 1, 1])
    assert out["rel_error"] <= 1e-13


def test_multigrid_reaches_the_fine_grid_als_result(orc):
    """From interpolated coarse subspaces, the sweeps on the finest grid reach
    the result of the same number of sweeps started from the fine grid's own
    HOSVD (E to 1e-6 relative, factors to small angles), and E is the fine
    HOSVD's or better."""
    k = orc.make_kernel(orc.MATERN, nu=0.8, ell=[0.3, 0.4, 0.5])
    g = orc.make_grid([32, 28, 24])
    rf = [5, 5, 4]
    mg = orc.multigrid(k, g, 1e-3, levels=2, sweeps=6, rfix=rf)
    fine = orc.hosvd(k, g, 1e-3, rfix=rf)
    F = orc.tensor(k, g)
    U, B, _ = orc.hooi(F, fine["U"], 6)
    e_als = orc.rel_error(F, orc.reconstruct(B, U, g.n))
    assert abs(mg["rel_error"] - e_als) <= 1e-6 * e_als
    assert mg["rel_error"] <= fine["rel_error"] * (1 + 1e-9)
    for a in range(3):
        s = np.linalg.svd(mg["U"][a] - U[a] @ (U[a].T @ mg["U"][a]), compute_uv=False)
        assert s.max() <= 1e-5


def test_multigrid_without_levels_is_hosvd_then_als(orc):
    k = orc.make_kernel(orc.MATERN, nu=1.3, ell=[0.3, 0.35, 0.4])
    g = orc.make_grid([12, 14, 16])
    mg = orc.multigrid(k, g, 1e-4, levels=0, sweeps=2, rmax=[6, 6, 6])
    ref = orc.hosvd(k, g, 1e-4, rmax=[6, 6, 6])
    U, B, _ = orc.hooi(orc.tensor(k, g), ref["U"], 2)
    assert mg["ranks"] == ref["ranks"]
    for a in range(3):
        assert np.array_equal(mg["U"][a], U[a])
    assert np.array_equal(mg["core"], B)


# ---- canonical-to-Tucker (Sec. 3.4) -----------------------------------------


def _cp():
    from paper_1711_06874_gb300 import cp_inputs

    return cp_inputs


def test_newton_sinc_cp_is_one_over_r(orc):
    """The sinc expansion of Eq. sinc_Newt with h_M = 3 log(M) / M, M = 64,
    reproduces 1/|x| at every grid point with |x| >= 0.5 (the quadrature's
    truncation and discretisation errors are both below 1e-13 there)."""
    cp = _cp()
    n = 24
    c, U = cp.newton_sinc_cp(n, 64)
    A = orc.cp_full(c, U)
    x = cp.grid_points(n)
    r = np.sqrt(x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2)
    far = r >= 0.5
    assert np.max(np.abs(A[far] * r[far] - 1.0)) <= 1e-13
    for u in U:
        np.testing.assert_allclose(np.linalg.norm(u, axis=0), 1.0, atol=1e-14)


def test_cp_norm_is_the_full_tensor_norm(orc):
    c, U = _cp().random_cp(3, (7, 8, 9), 6)
    assert abs(orc.cp_norm2(c, U) - orc.norm2(orc.cp_full(c, U))) <= 1e-13 * orc.norm2(orc.cp_full(c, U))


def test_rhosvd_core_is_the_projection_of_the_full_tensor(orc):
    """B formed in the canonical format equals the full tensor's TTM chain
    with the same factors (a dropped weight or a transposed W fails)."""
    c, U = _cp().random_cp(5, (9, 10, 11), 7)
    res = orc.rhosvd(c, U, 1e-3, rfix=[3, 4, 5])
    A = orc.cp_full(c, U)
    np.testing.assert_allclose(res["core"], orc.core(A, res["U"], res["ranks"]), rtol=0,
                               atol=1e-13 * math.sqrt(orc.norm2(A)))
    for l, z in enumerate(res["U"]):
        np.testing.assert_allclose(z.T @ z, np.eye(res["ranks"][l]), atol=1e-13)
        # the factors span the side matrix's leading left singular subspace
        Ul = np.linalg.svd(U[l])[0][:, : res["ranks"][l]]
        assert _principal_sines(Ul, z).max() <= 1e-12


def test_rhosvd_error_bound_and_eps_rule(orc):
    """|A - A_r| <= |c| sum_l sqrt(sum_{k > r_l} s_{l,k}^2) (the RHOSVD bound),
    for fixed ranks and for the eps rule, which then meets E <= eps."""
    c, U = _cp().random_cp(9, (12, 13, 14), 10)
    A = orc.cp_full(c, U)
    for kw in (dict(rfix=[3, 4, 5]), dict(rfix=[6, 2, 4])):
        res = orc.rhosvd(c, U, 1e-3, **kw)
        X = orc.reconstruct(res["core"], res["U"], A.shape)
        err = math.sqrt(orc.norm2(A - X))
        assert err <= res["bound"] * (1 + 1e-12)
        assert err > 0
    cs, Us = _cp().newton_sinc_cp(16, 12)
    As = orc.cp_full(cs, Us)
    for eps in (1e-3, 1e-6):
        res = orc.rhosvd(cs, Us, eps)
        X = orc.reconstruct(res["core"], res["U"], As.shape)
        assert orc.rel_error(As, X) <= eps
        assert res["bound"] <= eps * math.sqrt(res["normA2"]) * (1 + 1e-12)
        assert max(res["ranks"]) < 16


def test_rhosvd_exact_on_side_matrices_of_low_column_rank(orc):
    """Side matrices of column rank (2, 3, 4): those are the ranks at a tiny
    eps, and the Tucker tensor is exact; a rank-one CP tensor gives (1, 1, 1)."""
    c, U = _cp().random_cp(13, (10, 11, 12), 9, col_rank=(2, 3, 4))
    A = orc.cp_full(c, U)
    res = orc.rhosvd(c, U, 1e-10)
    assert res["ranks"] == [2, 3, 4]
    assert orc.rel_error(A, orc.reconstruct(res["core"], res["U"], A.shape)) <= 1e-13
    c1, U1 = _cp().random_cp(17, (6, 7, 8), 1)
    res1 = orc.rhosvd(c1, U1, 1e-12)
    assert res1["ranks"] == [1, 1, 1]
    assert abs(abs(res1["core"].item()) - abs(c1[0])) <= 1e-14 * abs(c1[0])


def test_c2t_sweeps_are_the_full_tensor_sweeps(orc):
    """The C2T sweeps in the canonical format give the factors, core and
    core-norm history of Tucker-ALS on the full tensor from the same start
    (the single-hole unfolding built from the side matrices is the full
    tensor's, up to a column order)."""
    cp = _cp()
    for c, U, rfix in (cp.newton_sinc_cp((14, 16, 18), 10) + ([4, 5, 6],),
                       cp.random_cp(21, (9, 10, 11), 8) + ([3, 4, 3],)):
        A = orc.cp_full(c, U)
        out = orc.c2t(c, U, 1e-3, 2, rfix=rfix)
        Uo, Bo, ho = orc.hooi(A, out["rhosvd"]["U"], 2)
        nA2 = orc.norm2(A)
        np.testing.assert_allclose(out["core_norm2_hist"], ho, rtol=0, atol=1e-12 * nA2)
        for l in range(3):
            assert _principal_sines(Uo[l], out["U"][l]).max() <= 1e-9
        np.testing.assert_allclose(out["core"], orc.core(A, out["U"], out["ranks"]), rtol=0,
                                   atol=1e-12 * math.sqrt(nA2))
        e = orc.rel_error(A, orc.reconstruct(out["core"], out["U"], A.shape))
        e0 = orc.rel_error(A, orc.reconstruct(out["rhosvd"]["core"], out["rhosvd"]["U"], A.shape))
        assert e <= e0 * (1 + 1e-9)


def test_rhosvd_bound_is_attained(orc):
    """A case where the RHOSVD bound holds with equality: modes 2 and 3 are
    exactly rank one, mode 1 has two unit columns at angle theta, and c is
    the side matrix's second right singular vector, so the discarded part is
    s_2 |c| exactly (an off-by-one in the discarded tail fails here)."""
    n, th = 5, 0.7
    rng = np.random.default_rng(23)
    u1 = np.zeros(n)
    u1[0] = 1.0
    u2 = np.zeros(n)
    u2[0], u2[1] = math.cos(th), math.sin(th)
    v = rng.standard_normal(6)
    w = rng.standard_normal(7)
    U = [np.stack([u1, u2], 1), np.stack([v, v], 1) / np.linalg.norm(v), np.stack([w, w], 1) / np.linalg.norm(w)]
    c = np.linalg.svd(U[0])[2][1].copy()  # unit vector
    res = orc.rhosvd(c, U, 0.0, rfix=[1, 1, 1])
    A = orc.cp_full(c, U)
    err = math.sqrt(orc.norm2(A - orc.reconstruct(res["core"], res["U"], A.shape)))
    s2 = math.sqrt(1.0 - math.cos(th))  # singular values of [u1 u2]: sqrt(1 +- cos theta)
    assert abs(err - s2) <= 1e-13
    assert abs(res["bound"] - s2) <= 1e-13


def test_rhosvd_eps_rule_shares_eps_over_three_modes(orc):
    """Side matrices with dense, geometrically decaying spectra (ratio 0.6):
    every mode's discarded part of the bound is within eps |A| / 3, which
    the next smaller rank would exceed, so the whole bound is within eps |A|."""
    rng = np.random.default_rng(29)
    c = np.abs(rng.standard_normal(30)) + 0.5
    U = []
    for _ in range(3):
        Q1 = np.linalg.qr(rng.standard_normal((30, 30)))[0]
        Q2 = np.linalg.qr(rng.standard_normal((30, 30)))[0]
        M = Q1 @ np.diag(0.6 ** np.arange(30)) @ Q2.T
        U.append(M / np.linalg.norm(M, axis=0))
    nA = math.sqrt(orc.cp_norm2(c, U))
    cn = float(np.linalg.norm(c))
    for eps in (1e-2, 1e-4):
        res = orc.rhosvd(c, U, eps)
        assert res["bound"] <= eps * nA * (1 + 1e-12)
        for l in range(3):
            s = np.linalg.svd(U[l], compute_uv=False)
            r = res["ranks"][l]
            assert 1 <= r < 30
            assert cn * math.sqrt(float((s[r:] ** 2).sum())) <= eps * nA / 3 * (1 + 1e-12)
            assert cn * math.sqrt(float((s[r - 1:] ** 2).sum())) > eps * nA / 3
