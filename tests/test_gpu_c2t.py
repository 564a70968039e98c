"""Canonical-to-Tucker (Sec. 3.4) through tk_c2t against the oracle's c2t.

The oracle takes the side matrices' and the single-hole unfoldings' left
singular vectors from LAPACK's SVD, the CUDA path from the eigenvectors of
their FP64 Grams, so factors are compared by principal angles on the leading
columns whose squared-singular-value gaps are resolved (within
max(1e-9, 100 u / gap), u = 2^-53), and the core, the core-norm history and E
to tolerances that cover the two roundings.  Ranks must be the oracle's
unless its discarded tail sits within a factor 1 +- 0.5 of the threshold.

E of the sweeps: a Gram squares the condition number, so the Gram route
resolves the smallest kept directions less well than the SVD route.  On the
sinc CP with ranks 11 to 14, exact eigenvectors of the exact FP64 Grams
(numpy's eigh in a host emulation) already give E of about 6e-9 where the SVD
route gives 4e-10 or 2e-13: E is compared to 1e-3 relative plus 1e-7 absolute
(a tenth of the smallest eps used here), and must meet eps itself.
"""
import math

import numpy as np
import pytest

from tests._util import U64, principal_sines

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_06874_gb300 import binding

    c = binding.Context(0)
    yield c
    c.close()


def _cp():
    from paper_1711_06874_gb300 import cp_inputs

    return cp_inputs


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _near_tail_threshold(U, c, normA2, eps, r):
    """The oracle's tail at r - 1 or r within x(1 +- 0.5) of eps |A| / (3 |c|)."""
    tol = eps * math.sqrt(normA2) / (3 * float(np.linalg.norm(c)))
    s = np.linalg.svd(U, compute_uv=False)
    for q in (r - 1, r):
        if 1 <= q <= s.size:
            t = math.sqrt(float((s[q:] ** 2).sum()))
            if 0.5 * tol <= t <= 1.5 * tol:
                return True
    return False


def _check(ctx, orc, c, U, eps, sweeps, rmax=None, rfix=None, e_rtol=1e-3, e_abs=1e-7):
    res, hist = ctx.c2t(_dev(c), [_dev(u) for u in U], eps, sweeps, rmax=rmax, rfix=rfix)
    ranks, flags = res.ranks
    ref = orc.c2t(c, U, eps, sweeps, rmax=rmax, rfix=rfix)
    if ranks != ref["ranks"]:
        for l in range(3):
            if ranks[l] != ref["ranks"][l]:
                assert abs(ranks[l] - ref["ranks"][l]) == 1
                assert _near_tail_threshold(U[l], c, ref["rhosvd"]["normA2"], eps, ref["ranks"][l]), l
        ref = orc.c2t(c, U, eps, sweeps, rfix=ranks)
    nA2 = orc.cp_norm2(c, U)
    assert abs(res.norm2 - nA2) <= 1e-13 * nA2
    Z = [res.factor(l) for l in range(3)]
    B = res.core()
    for l in range(3):
        np.testing.assert_allclose(Z[l].T @ Z[l], np.eye(ranks[l]), atol=1e-12)
    # B is the projection of A on the returned factors (canonical format)
    W = [Z[l].T @ U[l] for l in range(3)]
    np.testing.assert_allclose(B, orc.cp_core(c, W), rtol=0, atol=1e-12 * math.sqrt(nA2))
    # factors: principal angles on the resolved leading columns
    for l in range(3):
        if sweeps == 0:
            sv2 = np.linalg.svd(U[l], compute_uv=False) ** 2
        else:
            m, q = [a for a in range(3) if a != l]
            Wm, Wq = ref["U"][m].T @ U[m], ref["U"][q].T @ U[q]
            KR = (Wm[:, None, :] * Wq[None, :, :]).reshape(-1, c.size)
            sv2 = np.linalg.svd((U[l] * c[None, :]) @ KR.T, compute_uv=False) ** 2
        rp = 0
        for i in range(ranks[l]):
            if i + 1 < sv2.size and (sv2[i] - sv2[i + 1]) / sv2[0] >= 1e-6:
                rp = i + 1
            else:
                break
        if rp:
            gap = min((sv2[i] - sv2[i + 1]) / sv2[0] for i in range(rp))
            assert principal_sines(ref["U"][l][:, :rp], Z[l][:, :rp]).max() <= max(1e-9, 100 * U64 / gap), l
    if sweeps:
        np.testing.assert_allclose(hist, ref["core_norm2_hist"], rtol=0, atol=1e-9 * nA2)
        assert all(hist[i + 1] >= hist[i] - 1e-12 * nA2 for i in range(len(hist) - 1))
    # E by direct subtraction on the full tensor (small n)
    A = orc.cp_full(c, U)
    e = orc.rel_error(A, orc.reconstruct(B, Z, A.shape))
    e_o = orc.rel_error(A, orc.reconstruct(ref["core"], ref["U"], A.shape))
    assert abs(e - e_o) <= e_rtol * e_o + e_abs, (e, e_o)
    if rfix is None and not any(f & 1 for f in flags):
        # ranks from the eps rule (none capped): the RHOSVD bound gives E <= eps
        assert e <= eps * (1 + 1e-9)
    return res, ref, e


@pytest.mark.parametrize("sweeps", [0, 1, 2])
def test_c2t_newton_sinc_matches_oracle(ctx, orc, sweeps):
    """The paper's CP example: the sinc expansion of 1/|x| (Eq. sinc_Newt)."""
    c, U = _cp().newton_sinc_cp((32, 40, 48), 24)
    for eps in (1e-4, 1e-6):
        _check(ctx, orc, c, U, eps, sweeps)


def test_c2t_random_cp_fixed_ranks(ctx, orc):
    c, U = _cp().random_cp(21, (24, 30, 36), 40)
    _check(ctx, orc, c, U, 1e-3, 2, rfix=[5, 6, 7])


def test_c2t_exact_on_low_column_rank(ctx, orc):
    """Side matrices of column rank (2, 3, 4): the RHOSVD recovers the tensor."""
    c, U = _cp().random_cp(13, (10, 11, 12), 9, col_rank=(2, 3, 4))
    res, _, e = _check(ctx, orc, c, U, 1e-10, 1, e_abs=1e-12)
    assert res.ranks[0] == [2, 3, 4]
    assert e <= 1e-12
    # eps^2 |A|^2 / (9 |c|^2) lies below the FP64 Gram's rounding level
    # n_l u |U_l|^2: the discarded noise counts as zero, and the flag says so
    assert all(f & 2 for f in res.ranks[1])


def test_c2t_rank_cap_flag(ctx, orc):
    c, U = _cp().newton_sinc_cp((20, 20, 20), 16)
    res, _, _ = _check(ctx, orc, c, U, 1e-12, 1, rmax=[3, 3, 3])
    ranks, flags = res.ranks
    assert ranks == [3, 3, 3] and all(f & 1 for f in flags)


def test_c2t_rejects_bad_arguments(ctx):
    from paper_1711_06874_gb300 import binding

    c, U = _cp().newton_sinc_cp((8, 8, 8), 4)
    cd, Ud = _dev(c), [_dev(u) for u in U]
    for kw in (dict(eps=-1.0, sweeps=1), dict(eps=1e-3, sweeps=65), dict(eps=1e-3, sweeps=1, rmax=[97, 3, 3]),
               dict(eps=1e-3, sweeps=1, rfix=[-1, 0, 0])):
        with pytest.raises(binding.TuckerError) as ei:
            ctx.c2t(cd, Ud, **kw)
        assert ei.value.status == binding.TK_EINVAL
    # ranks that are not a multilinear rank
    with pytest.raises(binding.TuckerError) as ei:
        ctx.c2t(cd, Ud, 1e-3, 1, rfix=[5, 1, 1])
    assert ei.value.status == binding.TK_EINVAL
