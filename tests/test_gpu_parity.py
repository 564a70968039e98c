"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Every step of the hot path is compared element by element on the same seeded
inputs, at sizes the oracle finishes in seconds that span several 64-wide
tiles and a ragged tail; the whole solve is compared at the small Slater
configuration and at ragged anisotropic shapes.  Tolerances (FP64 path):
  tensor      |F - F_or| <= 5e-14 |F|_max     (K_nu to ~2e-15, grid rounding)
  Gram        |G - G_or| <= 1e-13 |G|_max     (FP64 sums of n^2 terms)
  eigen       |lam - lam_or| <= 1e-13 lam_1; principal angles on the leading
              columns whose gaps exceed 1e-6 lam_1 within max(1e-10, 10 u / gap),
              the Davis-Kahan bound for a Gram of unit roundoff u (2^-53 for
              the FP64 path, 2^-48 for the sliced Gram)
  core/recon  |B| to 1e-12 |F|; |X - X_or| <= max(1e-12, 100 u / eps) |F|
  ranks       equal, except when the oracle's discarded sum lies within a
              factor 1 +- 0.5 of the threshold (then +-1), or both are capped.
"""
import math

import numpy as np
import pytest

from tests._util import U64, angle_tol, compare_solution, principal_sines, separated_prefix

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


# ---------------------------------------------------------------------------
# (a) sampling
# ---------------------------------------------------------------------------
EVAL_CASES = [
    dict(kind=0, nu=1.2, ell=0.2, n=64),                      # table path, even n
    dict(kind=0, nu=0.5, ell=0.3, n=33),                      # table path, odd n
    dict(kind=0, nu=2.5, ell=0.1, n=40, grid=1),              # vertex grid, even n
    dict(kind=0, nu=0.3, ell=0.05, n=31, grid=1),             # vertex grid, odd n (r = 0 at centre)
    dict(kind=0, nu=1.7, ell=(0.2, 0.35, 0.5), n=(20, 24, 28)),  # general per-point path
    dict(kind=1, p=0.2, ell=1.0, n=24, b=5.0, grid=1),        # p-Slater
    dict(kind=2, ell=0.4, n=(17, 9, 30), b=(1.0, 0.5, 2.0)),  # Gaussian, non-cubic
    dict(kind=3, nu=0.4, p=0.1, n=40),                        # spectral density, table path
    dict(kind=3, nu=1.3, p=2.0, ell=(0.5, 0.8, 1.0), n=(20, 24, 28)),  # spectral density, general path
]


@pytest.mark.parametrize("case", EVAL_CASES)
def test_eval_matches_oracle(ctx, orc, wl, case):
    prob = wl.problem(**case)
    F = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    ctx.eval(prob, F)
    ref = orc.tensor(wl.oracle_kernel(prob, orc), wl.oracle_grid(prob, orc))
    got = F.cpu().numpy()
    assert np.abs(got - ref).max() <= 5e-14 * np.abs(ref).max()


# ---------------------------------------------------------------------------
# (b) Gram, all three unfoldings, ragged tiles
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(70, 45, 33), (64, 64, 64), (5, 130, 9), (2, 2, 2)])
def test_gram_fp64_matches_oracle(ctx, orc, shape):
    rng = np.random.default_rng(17)
    Fh = rng.random(shape)
    F = _dev(Fh)
    for mode in range(3):
        m = shape[mode]
        G = torch.empty((m, m), dtype=torch.float64, device="cuda")
        ctx.gram(F, mode, G)
        ref = orc.gram(Fh, mode)
        assert np.abs(G.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max(), mode


# ---------------------------------------------------------------------------
# (c) eigenpairs
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,m", [(64, 28), (130, 40), (48, 48), (97, 96), (9, 1)])
def test_sym_eig_matches_oracle(ctx, orc, wl, n, m):
    prob = wl.problem(0, nu=0.9, ell=0.25, n=(n, 20, 24))
    Fh = orc.tensor(wl.oracle_kernel(prob, orc), wl.oracle_grid(prob, orc))
    Gh = orc.gram(Fh, 0)
    lam_o, V_o, _ = orc.sym_eig(Gh)
    G = _dev(Gh)
    lam = torch.empty(m, dtype=torch.float64, device="cuda")
    V = torch.empty((n, m), dtype=torch.float64, device="cuda")
    ctx.sym_eig(G, m, lam, V)
    lam, V = lam.cpu().numpy(), V.cpu().numpy()
    np.testing.assert_allclose(lam, lam_o[:m], rtol=0, atol=1e-13 * lam_o[0])
    np.testing.assert_allclose(V.T @ V, np.eye(m), atol=1e-13)
    rp = min(separated_prefix(lam_o[:m]), m - 1 if m < n else m)
    for j in range(1, rp + 1):
        assert principal_sines(V_o[:, :j], V[:, :j]).max() <= 1e-10, j
    # canonical sign on separated columns
    for j in range(rp):
        assert np.dot(V[:, j], V_o[:, j]) > 0


# ---------------------------------------------------------------------------
# (d) core by chained TTMs
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,r", [((40, 48, 56), (5, 7, 9)), ((64, 64, 64), (11, 11, 11)),
                                     ((3, 70, 5), (1, 2, 5))])
def test_ttm_core_matches_oracle(ctx, orc, shape, r):
    rng = np.random.default_rng(5)
    Fh = rng.standard_normal(shape)
    U = [np.linalg.qr(rng.standard_normal((n, n)))[0][:, :k].copy() for n, k in zip(shape, r)]
    ref = orc.core(Fh, U, r)
    B = torch.empty(r, dtype=torch.float64, device="cuda")
    ctx.ttm_core(_dev(Fh), [_dev(u) for u in U], B)
    assert np.abs(B.cpu().numpy() - ref).max() <= 1e-13 * np.abs(Fh).max() * math.sqrt(Fh.size)


# ---------------------------------------------------------------------------
# Whole solve against the oracle
# ---------------------------------------------------------------------------
def _compare_solution(orc, wl, res, prob, precision_u=U64):
    return compare_solution(orc, wl, res, prob, precision_u)


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
def test_tucker_slater_n64_matches_oracle(ctx, orc, wl, eps):
    from paper_1711_06874_gb300 import binding

    prob = wl.slater_n64(eps)
    res = ctx.tucker(prob, precision=binding.TK_FP64)
    ref, e = _compare_solution(orc, wl, res, prob)
    if eps >= 1e-6:
        assert res.ranks[0] == ref["ranks"]
        assert e <= 2 * ref["rel_error"]


@pytest.mark.parametrize("case", [
    dict(nu=1.2, ell=(0.25, 0.3, 0.4), n=(40, 48, 70), eps=1e-6, rmax=24),
    dict(nu=2.5, ell=0.15, n=(33, 33, 33), eps=1e-5, rmax=16, grid=1),
    dict(nu=0.7, ell=0.2, n=(66, 66, 66), eps=1e-6, rmax=30),
])
def test_tucker_ragged_matches_oracle(ctx, orc, wl, case):
    from paper_1711_06874_gb300 import binding

    prob = wl.problem(0, **case)
    for shortcut in (True, False):
        res = ctx.tucker(prob, precision=binding.TK_FP64, shortcut=shortcut)
        _compare_solution(orc, wl, res, prob)


def test_gaussian_rank_one_on_gpu(ctx, wl):
    from paper_1711_06874_gb300 import binding

    prob = wl.problem(2, ell=0.4, n=48, eps=1e-6, rmax=8)
    res = ctx.tucker(prob, precision=binding.TK_FP64)
    assert res.ranks[0] == [1, 1, 1]
    assert res.rel_error() <= 1e-13


def test_full_rank_is_exact_on_gpu(ctx, wl):
    from paper_1711_06874_gb300 import binding

    prob = wl.problem(0, nu=0.5, ell=0.3, n=(12, 10, 14), eps=0.0, rmax=14)
    res = ctx.tucker(prob, precision=binding.TK_FP64, rfix=(12, 10, 14))
    assert res.ranks[0] == [12, 10, 14]
    assert res.rel_error() <= 1e-13
    assert abs(float(np.sum(res.core() ** 2)) - res.norm2) <= 1e-13 * res.norm2


def test_reconstruct_matches_oracle(ctx, orc, wl):
    from paper_1711_06874_gb300 import binding

    prob = wl.problem(0, nu=1.2, ell=0.2, n=(20, 30, 40), eps=1e-5, rmax=12)
    res = ctx.tucker(prob, precision=binding.TK_FP64)
    X = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    res.reconstruct(X)
    U = [res.factor(a) for a in range(3)]
    ref = orc.reconstruct(res.core(), U, prob.n)
    assert np.abs(X.cpu().numpy() - ref).max() <= 1e-14 * np.abs(ref).max()


def test_invalid_arguments_are_rejected(ctx, wl):
    from paper_1711_06874_gb300 import binding

    bad = [wl.problem(0, nu=0.0), wl.problem(0, ell=-1.0), wl.problem(0, n=1), wl.problem(0, eps=-1.0),
           wl.problem(0, rmax=0), wl.problem(0, rmax=89), wl.problem(0, n=2000)]
    for prob in bad:
        with pytest.raises(binding.TuckerError) as ei:
            ctx.tucker(prob, precision=binding.TK_FP64)
        assert ei.value.status == binding.TK_EINVAL


def test_fresh_context_per_shape(orc, wl):
    """Workspace sizing on a new context (no larger earlier reservation to hide behind)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_06874_gb300 import binding

    for case in [dict(nu=1.2, ell=(0.25, 0.3, 0.35), n=(24, 28, 32), eps=1e-6, rmax=16),
                 dict(nu=0.5, ell=0.3, n=(16, 16, 16), eps=1e-4, rmax=8)]:
        c = binding.Context(0)
        prob = wl.problem(0, **case)
        res = c.tucker(prob, precision=binding.TK_FP64)
        ref = orc.hosvd(wl.oracle_kernel(prob, orc), wl.oracle_grid(prob, orc), prob.eps, rmax=list(prob.rmax))
        assert res.ranks[0] == ref["ranks"]
        res.free()
        c.close()


def test_profile_and_launch_counter(ctx, wl):
    from paper_1711_06874_gb300 import binding

    prob = wl.problem(0, nu=1.2, ell=0.2, n=32, eps=1e-6, rmax=12)
    l0 = binding.Context.kernel_launches()
    ctx.profile(True)
    res = ctx.tucker(prob, precision=binding.TK_FP64)
    res.rel_error()
    prof = ctx.profile_read()
    ctx.profile(False)
    assert binding.Context.kernel_launches() > l0 + 5
    for stage in ("eval", "gram", "eig", "rank", "core", "error"):  # |F|^2 comes from trace(G)
        assert prof[stage][1] >= 1 and prof[stage][0] > 0.0, stage


# ---------------------------------------------------------------------------
# Mixed path: Gram from exact BF16 slices on the tcgen05 tensor cores
# ---------------------------------------------------------------------------
U_SLICED = 2.0 ** -48


@pytest.mark.parametrize("shape", [(70, 45, 33), (64, 64, 64), (200, 3, 5), (130, 9, 40), (2, 2, 2), (256, 16, 16)])
def test_gram_sliced_matches_oracle(ctx, orc, shape):
    from paper_1711_06874_gb300 import binding

    rng = np.random.default_rng(23)
    Fh = rng.random(shape) * np.exp(-3 * rng.random(shape))  # entries over about 1.3 decades
    F = _dev(Fh)
    for mode in range(3):
        m = shape[mode]
        G = torch.empty((m, m), dtype=torch.float64, device="cuda")
        ctx.gram(F, mode, G, precision=binding.TK_SLICED_BF16)
        ref = orc.gram(Fh, mode)
        got = G.cpu().numpy()
        # rigorous per-entry bound of the 6-slice scheme: each scaled entry is
        # exact to 2^-48 and the dropped weights add at most 5 2^-48, so
        # |dG_ij| <= 8 2^-48 K 2^(e_i + e_j) with 2^e_i > max_c |A(i, c)|
        A = np.moveaxis(Fh, mode, 0).reshape(m, -1)
        e = np.frexp(np.abs(A).max(axis=1))[1].astype(np.float64)
        bound = 8 * 2.0 ** -48 * A.shape[1] * np.exp2(e[:, None] + e[None, :])
        assert (np.abs(got - ref) <= bound).all(), (shape, mode, np.abs(got - ref).max())
        if A.shape[1] >= 256:  # with many terms the errors average out
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), (shape, mode)


def test_gram_sliced_exact_on_integer_grid(ctx):
    """Entries with few significant bits are represented exactly by the slices."""
    from paper_1711_06874_gb300 import binding

    rng = np.random.default_rng(3)
    Fh = rng.integers(-1000, 1000, size=(96, 40, 50)).astype(np.float64)
    F = _dev(Fh)
    for mode in range(3):
        A = np.moveaxis(Fh, mode, 0).reshape(Fh.shape[mode], -1).astype(np.int64)
        exact = (A @ A.T).astype(np.float64)
        G = torch.empty(exact.shape, dtype=torch.float64, device="cuda")
        ctx.gram(F, mode, G, precision=binding.TK_SLICED_BF16)
        np.testing.assert_array_equal(G.cpu().numpy(), exact)


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
def test_tucker_sliced_slater_n64_matches_oracle(ctx, orc, wl, eps):
    from paper_1711_06874_gb300 import binding

    prob = wl.slater_n64(eps)
    res = ctx.tucker(prob, precision=binding.TK_SLICED_BF16)
    ref, e = _compare_solution(orc, wl, res, prob, precision_u=U_SLICED)
    assert e <= 2 * ref["rel_error"] or res.ranks[1][0]


@pytest.mark.parametrize("case", [
    dict(nu=1.2, ell=(0.25, 0.3, 0.4), n=(40, 48, 70), eps=1e-6, rmax=24),
    dict(nu=0.7, ell=0.2, n=(66, 66, 66), eps=1e-6, rmax=30),
    dict(nu=2.5, ell=0.1, n=(130, 20, 24), eps=1e-5, rmax=24),
])
def test_tucker_sliced_ragged_matches_oracle(ctx, orc, wl, case):
    from paper_1711_06874_gb300 import binding

    prob = wl.problem(0, **case)
    res = ctx.tucker(prob, precision=binding.TK_SLICED_BF16)
    ref, e = _compare_solution(orc, wl, res, prob, precision_u=U_SLICED)
    assert e <= 2 * ref["rel_error"]


def test_tucker_bench_workload_full_size(ctx, orc, wl):
    """The benchmark's n = 256 workload in its launch configuration, both paths,
    against the oracle.  FP64 path: the small cases' bar (compare_solution:
    ranks, |F|^2, core norm, |X - X_or| <= max(1e-12, 100 u / eps) |F|,
    principal angles in all three modes, E of the GPU's factors), plus the
    eigenvalues to 1e-13 lam_1.  Sliced path: the same with u = 2^-48 and
    E <= 2 E_oracle."""
    from paper_1711_06874_gb300 import binding

    prob = wl.matern_n256(1e-6)
    ref = orc.hosvd(wl.oracle_kernel(prob, orc), wl.oracle_grid(prob, orc), prob.eps, rmax=list(prob.rmax))
    for precision in (binding.TK_FP64, binding.TK_SLICED_BF16):
        res = ctx.tucker(prob, precision=precision)
        ranks, _ = res.ranks
        assert ranks == ref["ranks"], (precision, ranks, ref["ranks"])
        u = U64 if precision == binding.TK_FP64 else U_SLICED
        _, e = compare_solution(orc, wl, res, prob, precision_u=u, ref=ref)
        assert e <= prob.eps and e <= 2 * ref["rel_error"], (precision, e, ref["rel_error"])
        if precision == binding.TK_FP64:
            # both FP64 routes take the factors from a Gram of rounding ~u lam_1:
            # E agrees to second order in the subspace error
            assert abs(e - ref["rel_error"]) <= 1e-2 * ref["rel_error"], (e, ref["rel_error"])
        for a in range(3):
            lam = res.eigenvalues(a)
            k = min(len(lam), ranks[a] + 2)
            np.testing.assert_allclose(lam[:k], ref["lam"][a][:k], rtol=0, atol=1e-13 * ref["lam"][a][0])
        res.free()
