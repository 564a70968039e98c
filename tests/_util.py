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
