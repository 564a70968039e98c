"""Helpers shared by the GPU parity tests (comparison measures only)."""
import numpy as np

U64 = 2.0 ** -53


def principal_sines(U, W):
    """Sines of the principal angles between span(U) and span(W) (orthonormal columns)."""
    return np.linalg.svd(W - U @ (U.T @ W), compute_uv=False)


def separated_prefix(lam, rel_gap=1e-6):
    """Largest r' such that every gap (lam_i - lam_{i+1}) / lam_1, i < r', is >= rel_gap."""
    lam = np.asarray(lam)
    r = 0
    for i in range(len(lam) - 1):
        if (lam[i] - lam[i + 1]) / lam[0] >= rel_gap:
            r = i + 1
        else:
            break
    return r


def near_threshold(lam_all, normF2, eps, r):
    """True when the oracle's discarded sum at r or r-1 is within x(1 +- 0.5) of the threshold."""
    thr = eps * eps * normF2 / 3.0
    lam = np.clip(np.asarray(lam_all), 0, None)

    def disc(q):
        return lam[q:].sum()

    for q in (r - 1, r):
        if 1 <= q <= len(lam) and 0.5 * thr <= disc(q) <= 1.5 * thr:
            return True
    return False


def angle_tol(lam, rp, precision_u):
    """1e-10, or the Davis-Kahan bound sin(theta) <= |dG| / gap when that is
    larger: a Gram of unit roundoff u is off by |dG| ~ 10 u lam_1, so the
    leading vectors are fixed only to 10 u / (smallest relative gap of the first
    rp eigenvalues) by the matrix itself (the oracle's too).  For the FP64 path
    this exceeds 1e-10 only for gaps below 1.1e-5 lam_1."""
    lam = np.asarray(lam)
    gap = min((lam[i] - lam[i + 1]) / lam[0] for i in range(rp))
    return max(1e-10, 10 * precision_u / gap)


def compare_solution(orc, wl, res, prob, precision_u=U64, ref=None):
    """A GPU result against the oracle's HOSVD of the same problem: ranks
    (equal unless both capped, both flagged, or the oracle's discarded sum at a
    threshold), |F|^2 to 1e-13, orthonormal factors, the core norm to 1e-12 |F|,
    the reconstruction to max(1e-12, 100 u / eps) |F|, principal angles of the
    separated leading columns in every mode, and E of the GPU's factors against
    the oracle's E of the same factors to 1e-10 relative."""
    import math

    kern, grid = wl.oracle_kernel(prob, orc), wl.oracle_grid(prob, orc)
    if ref is None:
        ref = orc.hosvd(kern, grid, prob.eps, rmax=list(prob.rmax))
    ranks, flags = res.ranks
    for a in range(3):
        if ranks[a] != ref["ranks"][a]:
            both_capped = ranks[a] == prob.rmax[a] and ref["ranks"][a] == prob.rmax[a]
            ok = (abs(ranks[a] - ref["ranks"][a]) <= 1
                  and near_threshold(ref["lam"][a], ref["normF2"], prob.eps, ref["ranks"][a]))
            assert both_capped or ok or (ref["flags"][a] & 2 and flags[a] & 2), (a, ranks, ref["ranks"])
    F = orc.tensor(kern, grid)
    nF = math.sqrt(ref["normF2"])
    assert abs(res.norm2 - ref["normF2"]) <= 1e-13 * ref["normF2"]
    U = [res.factor(a) for a in range(3)]
    B = res.core()
    for a in range(3):
        np.testing.assert_allclose(U[a].T @ U[a], np.eye(ranks[a]), atol=1e-13)
    if ranks == ref["ranks"]:
        assert abs(np.linalg.norm(B) - math.sqrt(ref["core_norm2"])) <= 1e-12 * nF
        X = orc.reconstruct(B, U, prob.n)
        Xo = orc.reconstruct(ref["core"], ref["U"], prob.n)
        tol = max(1e-12, 100 * precision_u / max(prob.eps, 1e-300))
        assert np.linalg.norm(X - Xo) <= tol * nF
        for a in range(3):
            rp = min(separated_prefix(ref["lam"][a][: ranks[a] + 1]), ranks[a])
            if rp:
                tol_a = angle_tol(ref["lam"][a], rp, precision_u)
                assert principal_sines(ref["U"][a][:, :rp], U[a][:, :rp]).max() <= tol_a
    # E: GPU rel_error (direct subtraction on the device) vs the oracle's on the GPU factors
    e_gpu = res.rel_error()
    e_or = orc.rel_error(F, orc.reconstruct(B, U, prob.n))
    assert abs(e_gpu - e_or) <= 1e-10 * e_or + 1e-15
    if not any(flags):
        assert e_gpu <= prob.eps * (1 + 1e-6)
    return ref, e_gpu
