"""Tucker-ALS (Sec. 3.2) through tk_als against the oracle's sweeps.

Both sides start from the same factors (the oracle's HOSVD, or a seeded
random orthonormal block) and run the same number of sweeps.  The oracle
takes each update from the one-sided Jacobi SVD of the single-hole
unfolding, the CUDA path from the eigenvectors of that unfolding's FP64
Gram, so factors are compared by principal angles and the core norms and E
to tolerances that cover the different roundings.
"""
import math

import numpy as np
import pytest

from tests._util import principal_sines

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


@pytest.fixture(scope="module")
def wl():
    from paper_1711_06874_gb300 import workloads

    return workloads


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _orthonormal(rng, n, r):
    q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return q


def _run(ctx, F, U0, sweeps):
    Fd = _dev(F)
    Ud = [_dev(u) for u in U0]
    r = [u.shape[1] for u in U0]
    Bd = torch.empty(r, dtype=torch.float64, device="cuda")
    hist = ctx.als(Fd, Ud, Bd, sweeps)
    return [u.cpu().numpy() for u in Ud], Bd.cpu().numpy(), hist


ALS_CASES = [
    dict(kind=0, nu=0.7, ell=(0.3, 0.5, 0.8), p=1.0, n=(20, 24, 28), r=(5, 4, 3), sweeps=3),
    dict(kind=1, nu=0.5, ell=(0.4, 0.4, 0.4), p=1.5, n=(17, 17, 17), r=(6, 6, 6), sweeps=2),
    dict(kind=3, nu=0.4, ell=(1.0, 1.0, 1.0), p=1.0, n=(16, 18, 20), r=(4, 4, 4), sweeps=2),
    dict(kind=0, nu=2.5, ell=(0.2, 0.25, 0.3), p=1.0, n=(48, 40, 36), r=(9, 8, 7), sweeps=2),
]


@pytest.mark.parametrize("case", ALS_CASES, ids=lambda c: f"kind{c['kind']}-n{c['n'][0]}-r{c['r'][0]}")
def test_als_matches_oracle(ctx, orc, case):
    k = orc.make_kernel(case["kind"], nu=case["nu"], ell=list(case["ell"]), p=case["p"])
    g = orc.make_grid(list(case["n"]), b=[1.0, 1.0, 1.0])
    F = orc.tensor(k, g)
    ref = orc.hosvd(k, g, 1e-3, rfix=list(case["r"]))
    nF2 = ref["normF2"]
    Uo, Bo, ho = orc.hooi(F, ref["U"], case["sweeps"])
    U, B, h = _run(ctx, F, ref["U"], case["sweeps"])
    assert h.shape == ho.shape
    np.testing.assert_allclose(h, ho, rtol=0, atol=1e-9 * nF2)
    assert np.all(np.diff(h) >= -1e-12 * nF2)
    for a in range(3):
        np.testing.assert_allclose(U[a].T @ U[a], np.eye(case["r"][a]), atol=1e-12)
        # the last update's Gram is off by about 10 u lam_1 (it squares the
        # unfolding, the oracle's SVD does not), which fixes its leading
        # vectors only to 10 u lam_1 / gap (Davis-Kahan); the factor 100
        # covers the carry-over from the earlier updates of the sweeps
        m1, m2 = [b for b in range(3) if b != a]
        Y = orc.ttm(orc.ttm(F, m1, Uo[m1]), m2, Uo[m2])
        lam = orc.unfolding_svd(Y, a)[0] ** 2
        ra = case["r"][a]
        gap = min((lam[i] - lam[i + 1]) / lam[0] for i in range(ra))
        assert principal_sines(Uo[a], U[a]).max() <= max(1e-9, 100 * 2.0 ** -53 / gap), (a, gap)
    # B is the core of the returned factors
    np.testing.assert_allclose(B, orc.core(F, U, case["r"]), rtol=0, atol=1e-12 * math.sqrt(nF2))
    e = orc.rel_error(F, orc.reconstruct(B, U, case["n"]))
    e_o = orc.rel_error(F, orc.reconstruct(Bo, Uo, case["n"]))
    assert abs(e - e_o) <= 1e-6 * e_o + 1e-14
    assert e <= ref["rel_error"] * (1 + 1e-9)


def test_als_zero_sweeps_is_the_core(ctx, orc):
    k = orc.make_kernel(orc.MATERN, nu=1.1, ell=[0.3, 0.4, 0.5])
    g = orc.make_grid([13, 15, 17], b=[1.0, 1.0, 1.0])
    F = orc.tensor(k, g)
    rng = np.random.default_rng(5)
    U0 = [_orthonormal(rng, n, r) for n, r in zip((13, 15, 17), (3, 5, 4))]
    U, B, h = _run(ctx, F, U0, 0)
    assert h.size == 0
    for a in range(3):
        assert np.array_equal(U[a], U0[a])
    np.testing.assert_allclose(B, orc.core(F, U0, (3, 5, 4)), rtol=0, atol=1e-13 * np.linalg.norm(F))


def test_als_rank_one_gaussian_is_a_fixed_point(ctx, orc):
    k = orc.make_kernel(orc.GAUSSIAN, ell=[0.4, 0.6, 0.9])
    g = orc.make_grid([10, 11, 12], b=[1.0, 1.0, 1.0])
    F = orc.tensor(k, g)
    ref = orc.hosvd(k, g, 1e-3, rfix=[1, 1, 1])
    U, B, h = _run(ctx, F, ref["U"], 2)
    for a in range(3):
        np.testing.assert_allclose(U[a], ref["U"][a], rtol=0, atol=1e-13)
    assert orc.rel_error(F, orc.reconstruct(B, U, g.n)) <= 1e-13


def test_als_recovers_exact_multilinear_rank_from_random_start(ctx, orc):
    rng = np.random.default_rng(11)
    n, r = (40, 36, 33), (3, 4, 2)
    G = rng.standard_normal(r)
    Q = [_orthonormal(rng, n[a], r[a]) for a in range(3)]
    F = np.einsum("abc,ia,jb,kc->ijk", G, *Q)
    U0 = [_orthonormal(rng, n[a], r[a]) for a in range(3)]
    U, B, h = _run(ctx, F, U0, 1)
    assert orc.rel_error(F, orc.reconstruct(B, U, n)) <= 1e-12
    assert abs(h[-1] - orc.norm2(F)) <= 1e-12 * orc.norm2(F)
    for a in range(3):
        assert principal_sines(Q[a], U[a]).max() <= 1e-10


def test_als_rejects_a_non_multilinear_rank(ctx):
    F = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
    U = [torch.zeros((8, r), dtype=torch.float64, device="cuda") for r in (1, 1, 3)]
    B = torch.empty((1, 1, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        ctx.als(F, U, B, 1)


def test_als_bench_workload_full_size(ctx, orc, wl):
    """The n = 256 Matern workload (nu = 1.2, ell = 0.2, eps = 1e-6) from the
    FP64 HOSVD's factors, in the launch configuration the benchmark's ALS
    workload times: the history is monotone and starts at or above the HOSVD
    core norm, the factors stay orthonormal, B is the oracle's core of the
    returned factors, and E does not exceed the HOSVD's."""
    from paper_1711_06874_gb300 import binding

    prob = wl.matern_n256(1e-6)
    res = ctx.tucker(prob, precision=binding.TK_FP64)
    ranks, _ = res.ranks
    U0 = [res.factor(a) for a in range(3)]
    Fd = torch.empty(tuple(prob.n), dtype=torch.float64, device="cuda")
    ctx.eval(prob, Fd)
    Ud = [_dev(u) for u in U0]
    Bd = torch.empty(ranks, dtype=torch.float64, device="cuda")
    hist = ctx.als(Fd, Ud, Bd, 2)
    U = [u.cpu().numpy() for u in Ud]
    B = Bd.cpu().numpy()
    F = orc.tensor(wl.oracle_kernel(prob, orc), wl.oracle_grid(prob, orc))
    nF2 = orc.norm2(F)
    assert hist[0] >= np.linalg.norm(res.core()) ** 2 - 1e-12 * nF2
    assert np.all(np.diff(hist) >= -1e-12 * nF2)
    for a in range(3):
        np.testing.assert_allclose(U[a].T @ U[a], np.eye(ranks[a]), atol=1e-12)
    np.testing.assert_allclose(B, orc.core(F, U, ranks), rtol=0, atol=1e-12 * math.sqrt(nF2))
    e = orc.rel_error(F, orc.reconstruct(B, U, prob.n))
    e_h = orc.rel_error(F, orc.reconstruct(res.core(), U0, prob.n))
    assert e <= e_h * (1 + 1e-6), (e, e_h)
