"""Batched solves (tk_batch) and the folded solve, through the C-ABI.

  * fold vs whole tensor: the weighted-octant solve gives the ranks,
    eigenvalues (to 1e-13 lam_1), factors (principal angles) and core norm of
    the unfolded one;
  * a batch against each instance alone: bitwise equal ranks, flags,
    eigenvalues, |F|^2, factors and cores, for a mix of shapes, grids,
    tolerances and both precisions (rank groups, escalation to all pairs);
  * a batch against the oracle, small instances element by element;
  * the 256-instance n = 128 parameter sweep at full size: sampled instances
    against the oracle, every instance for orthonormal factors, the HOSVD
    bound and its rel_error;
  * repeated solves of one plan (run plainly, captured into a CUDA graph,
    replayed, recaptured after the workspaces moved): bitwise the same
    results and the same kernel count every time.
"""
import math

import numpy as np
import pytest

from tests._util import U64, near_threshold, principal_sines, separated_prefix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U_SLICED = 2.0 ** -48


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


def _same(a, b):
    return a.shape == b.shape and np.array_equal(a, b)


FOLD_CASES = [
    dict(nu=1.2, ell=0.2, n=48, eps=1e-6, rmax=20),
    dict(nu=0.7, ell=(0.25, 0.3, 0.4), n=(40, 33, 27), eps=1e-6, rmax=24),
    dict(nu=2.5, ell=0.15, n=35, eps=1e-5, rmax=16, grid=1),
    dict(nu=0.4, ell=0.08, n=(30, 31, 32), eps=1e-4, rmax=30, grid=1),
]


@pytest.mark.parametrize("case", FOLD_CASES)
def test_fold_matches_whole_tensor(ctx, wl, case):
    from paper_1711_06874_gb300 import binding

    prob = wl.problem(0, **case)
    for precision, u in ((binding.TK_FP64, U64), (binding.TK_SLICED_BF16, U_SLICED)):
        rf = ctx.tucker(prob, precision=precision, fold=True)
        rw = ctx.tucker(prob, precision=precision, fold=False)
        assert rf.ranks == rw.ranks
        r = rf.ranks[0]
        assert abs(rf.norm2 - rw.norm2) <= 1e-14 * rw.norm2
        for a in range(3):
            lf, lw = rf.eigenvalues(a), rw.eigenvalues(a)
            k = min(len(lf), len(lw), r[a] + 1)
            # two FP64 sums of about n^2 terms each (the octant's are scaled by sqrt 2)
            np.testing.assert_allclose(lf[:k], lw[:k], rtol=0, atol=1e-12 * lw[0])
            Uf, Uw = rf.factor(a), rw.factor(a)
            np.testing.assert_allclose(Uf.T @ Uf, np.eye(r[a]), atol=1e-13)
            rp = min(separated_prefix(lw[: r[a] + 1]), r[a])
            if rp:
                gap = min((lw[i] - lw[i + 1]) / lw[0] for i in range(rp))
                tol = max(1e-10, 10 * u / gap) if u > U64 else 1e-10
                assert principal_sines(Uw[:, :rp], Uf[:, :rp]).max() <= tol
                # canonical signs agree on separated columns
                for j in range(rp):
                    assert np.dot(Uf[:, j], Uw[:, j]) > 0
        nB = np.linalg.norm(rw.core())
        assert abs(np.linalg.norm(rf.core()) - nB) <= 1e-12 * math.sqrt(rw.norm2)
        # factors from two roundings of G differ at first order only inside the
        # kept and the discarded subspaces; the error moves at second order
        assert abs(rf.rel_error() - rw.rel_error()) <= 1e-4 * rw.rel_error() + 1e-14


def _mix(wl):
    P = wl.problem
    return [
        P(0, nu=1.2, ell=0.2, n=40, eps=1e-6, rmax=20),
        P(0, nu=1.2, ell=0.2, n=40, eps=1e-10, rmax=20),      # eps below the Gram's precision
        P(0, nu=2.1, ell=0.9, n=40, eps=1e-6, rmax=20),       # low rank
        P(0, nu=1.2, ell=0.2, n=40, eps=1e-4, rmax=20),
        P(0, nu=0.8, ell=0.3, n=33, eps=1e-6, rmax=20, grid=1),
        P(0, nu=0.8, ell=(0.3, 0.4, 0.5), n=(20, 24, 28), eps=1e-6, rmax=12),
        P(0, nu=1.2, ell=0.2, n=40, eps=1e-6, rmax=20),       # duplicate of the first
        P(0, nu=0.3, ell=0.5, n=64, eps=1e-8, rmax=24),
        P(0, nu=1.0, ell=0.3, n=40, eps=1e-6, rmax=20),       # fixed rank 18 (below)
        P(0, nu=0.6, ell=0.15, n=40, eps=1e-8, rmax=20),
    ]


@pytest.mark.parametrize("precision_name", ["TK_FP64", "TK_SLICED_BF16"])
def test_batch_equals_alone_bitwise(ctx, wl, precision_name):
    from paper_1711_06874_gb300 import binding

    precision = getattr(binding, precision_name)
    probs = _mix(wl)
    rfixes = [(18, 18, 18) if i == 8 else (0, 0, 0) for i in range(len(probs))]
    mixed = ctx.batch(probs, precision=precision, rfixes=rfixes)
    for p, rf, rm in zip(probs, rfixes, mixed):
        (ra,) = ctx.batch([p], precision=precision, rfixes=[rf])
        rt = ctx.tucker(p, precision=precision, rfix=rf)
        for alone in (ra, rt):
            assert rm.ranks == alone.ranks
            assert rm.norm2 == alone.norm2
            assert _same(rm.core(), alone.core())
            for a in range(3):
                assert _same(rm.factor(a), alone.factor(a)), a
                assert _same(rm.eigenvalues(a), alone.eigenvalues(a)), a
    # the duplicate instance is bitwise the first
    assert _same(mixed[0].core(), mixed[6].core())
    assert mixed[8].ranks[0] == [18, 18, 18]  # fixed rank above the first pass: all pairs


def test_batch_matches_oracle(ctx, orc, wl):
    from paper_1711_06874_gb300 import binding

    probs = [wl.problem(0, nu=nu, ell=ell, n=36, eps=1e-6, rmax=24)
             for nu, ell in ((0.5, 0.3), (1.2, 0.2), (2.5, 0.5), (0.9, 0.1))]
    res = ctx.batch(probs, precision=binding.TK_FP64)
    for p, r in zip(probs, res):
        ref = orc.hosvd(wl.oracle_kernel(p, orc), wl.oracle_grid(p, orc), p.eps, rmax=list(p.rmax))
        ranks, _ = r.ranks
        assert ranks == ref["ranks"] or any(near_threshold(ref["lam"][a], ref["normF2"], p.eps, ref["ranks"][a])
                                            for a in range(3))
        if ranks != ref["ranks"]:
            continue
        nF = math.sqrt(ref["normF2"])
        assert abs(r.norm2 - ref["normF2"]) <= 1e-13 * ref["normF2"]
        B = r.core()
        assert abs(np.linalg.norm(B) - math.sqrt(ref["core_norm2"])) <= 1e-12 * nF
        U = [r.factor(a) for a in range(3)]
        X = orc.reconstruct(B, U, p.n)
        Xo = orc.reconstruct(ref["core"], ref["U"], p.n)
        # subspaces from two roundings of G: first order in u / eps
        assert np.linalg.norm(X - Xo) <= max(1e-12, 100 * U64 / p.eps) * nF
        e_or = orc.rel_error(orc.tensor(wl.oracle_kernel(p, orc), wl.oracle_grid(p, orc)), X)
        assert abs(r.rel_error() - e_or) <= 1e-10 * e_or + 1e-15


def test_batch_empty_and_invalid(ctx, wl):
    from paper_1711_06874_gb300 import binding

    assert ctx.batch([]) == []
    with pytest.raises(binding.TuckerError) as ei:
        ctx.batch([wl.problem(0, nu=1.0, n=16), wl.problem(0, nu=-1.0, n=16)])
    assert ei.value.status == binding.TK_EINVAL


def test_sweep_256_n128_full_size(ctx, orc, wl):
    """The 256-instance n = 128 sweep in one tk_batch call, mixed precision."""
    from paper_1711_06874_gb300 import binding

    probs = wl.sweep()
    res = ctx.batch(probs, precision=binding.TK_SLICED_BF16)
    assert len(res) == 256
    for p, r in zip(probs, res):
        ranks, flags = r.ranks
        lam = r.eigenvalues(0)
        U = r.factor(0)
        np.testing.assert_allclose(U.T @ U, np.eye(ranks[0]), atol=1e-12)
        # HOSVD: |B|^2 = |F|^2 - discarded, and the error below the bound
        e = r.rel_error()
        if not (flags[0] & binding.TK_RANK_CAPPED):
            assert e <= p.eps * (1 + 1e-6) or flags[0] & 2, (p, e)
    for i in (0, 97, 255):  # sampled instances against the oracle
        p, r = probs[i], res[i]
        ref = orc.hosvd(wl.oracle_kernel(p, orc), wl.oracle_grid(p, orc), p.eps, rmax=list(p.rmax))
        ranks, _ = r.ranks
        assert ranks == ref["ranks"] or near_threshold(ref["lam"][0], ref["normF2"], p.eps, ref["ranks"][0])
        assert abs(r.norm2 - ref["normF2"]) <= 1e-13 * ref["normF2"]
        k = min(len(r.eigenvalues(0)), ranks[0] + 1)
        np.testing.assert_allclose(r.eigenvalues(0)[:k], ref["lam"][0][:k], rtol=0, atol=1e-13 * ref["lam"][0][0])
        if ranks == ref["ranks"]:
            nF = math.sqrt(ref["normF2"])
            assert abs(np.linalg.norm(r.core()) - math.sqrt(ref["core_norm2"])) <= 1e-12 * nF


def test_error_during_solve(ctx, wl):
    """E from the overlapped second sampling equals tk_rel_error's, alone and in a batch."""
    from paper_1711_06874_gb300 import binding

    probs = [wl.problem(0, nu=nu, ell=ell, n=n, eps=1e-6, rmax=24)
             for nu, ell, n in ((1.2, 0.2, 48), (0.5, 0.3, 40), (2.0, 0.6, 48), (0.8, (0.3, 0.4, 0.5), (20, 24, 28)))]
    for precision in (binding.TK_FP64, binding.TK_SLICED_BF16):
        # FP64: the same FP64 arithmetic as tk_rel_error.  Sliced, isotropic:
        # the residual against the Gram's slices in float-float arithmetic
        # (about 2^-23 of each residual entry) and squares summed in FP32 over
        # at most 8 + 7 rounding steps before FP64, so |F - X|^2 carries about
        # 1e-6 of itself: 1e-5 on the relative error leaves a margin.
        tol = 1e-10 if precision == binding.TK_FP64 else 1e-5
        mixed = ctx.batch(probs, precision=precision, with_error=True)
        for p, rm in zip(probs, mixed):
            e_ref = rm.rel_error()
            assert abs(rm.solve_error - e_ref) <= tol * e_ref, (p, rm.solve_error, e_ref)
            alone = ctx.tucker(p, precision=precision, with_error=True)
            assert alone.solve_error == rm.solve_error
            assert np.array_equal(alone.core(), rm.core())
        plain = ctx.tucker(probs[0], precision=precision)
        with pytest.raises(binding.TuckerError):
            plain.solve_error


def test_repeated_solves_replay_bitwise(ctx, wl):
    """A small solve seen before runs as one CUDA graph (captured on its second
    run, replayed after): every result is bitwise the plain run's, the kernel
    count is the same, and a solve whose workspaces moved (a larger solve in
    between grows them) is run plainly and captured again."""
    from paper_1711_06874_gb300 import binding

    cases = [
        (wl.problem(0, nu=1.2, ell=0.2, n=48, eps=1e-6, rmax=24), binding.TK_SLICED_BF16, True, (0, 0, 0)),
        (wl.problem(0, nu=0.5, ell=0.3, n=40, eps=1e-6, rmax=24), binding.TK_FP64, False, (0, 0, 0)),
        (wl.problem(0, nu=0.8, ell=(0.3, 0.4, 0.5), n=(20, 24, 28), eps=1e-6, rmax=24), binding.TK_FP64, False,
         (0, 0, 0)),
        # a fixed rank above the first pass's 12 pairs (the eps rule reaches
        # such ranks on these grids only at the FP64 floor, where rounding
        # decides them): more pairs are computed the ordinary way every time
        (wl.problem(0, nu=0.6, ell=0.15, n=40, eps=1e-6, rmax=20), binding.TK_FP64, False, (14, 14, 14)),
    ]
    for i, (p, prec, we, rf) in enumerate(cases):
        big = wl.problem(0, nu=1.2, ell=0.2, n=160 + 32 * i, eps=1e-6, rmax=24)  # larger each case
        runs = []
        for k in range(7):
            if k == 4:
                ctx.tucker(big, precision=prec, with_error=we).free()  # grows the workspaces
            l0 = binding.Context.kernel_launches()
            r = ctx.tucker(p, precision=prec, rfix=rf, with_error=we)
            runs.append((r, binding.Context.kernel_launches() - l0))
        r0, k0 = runs[0]
        if rf[0] > 0:
            assert r0.ranks[0] == list(rf)
        for r, k in runs[1:]:
            assert k == k0
            assert r.ranks == r0.ranks
            assert r.norm2 == r0.norm2
            assert _same(r.core(), r0.core())
            for a in range(3):
                assert _same(r.factor(a), r0.factor(a)), a
                assert _same(r.eigenvalues(a), r0.eigenvalues(a)), a
            if we:
                assert r.solve_error == r0.solve_error


def test_result_copy_matches_accessors(ctx, wl):
    """tk_result_copy (one staged copy of U_1, U_2, U_3 and B) gives the bytes
    tk_factor and tk_core give: for a folded solve, for instances of a batch
    sharing one device block, and for an unfolded solve whose parts are
    separate allocations."""
    from paper_1711_06874_gb300 import binding

    probs = [wl.problem(0, nu=1.2, ell=0.2, n=48, eps=1e-6, rmax=24),
             wl.problem(0, nu=0.8, ell=(0.3, 0.4, 0.5), n=(20, 24, 28), eps=1e-6, rmax=24)]
    results = list(ctx.batch(probs, precision=binding.TK_SLICED_BF16))
    results.append(ctx.tucker(probs[0], precision=binding.TK_FP64, fold=False))
    for r in results:
        U1, U2, U3, B = r.factors_and_core()
        for a, U in enumerate((U1, U2, U3)):
            assert _same(U, r.factor(a)), a
        assert _same(B, r.core())


@pytest.mark.parametrize("precision_name", ["TK_FP64", "TK_SLICED_BF16"])
def test_spectral_density_matches_oracle(ctx, orc, wl, precision_name):
    """The spectral density of Eq. (SD_matern) through the whole solve (the
    paper's alpha = 0.1 and alpha = 100 with nu = 0.4, and a middle case):
    ranks as the oracle's unless at a threshold, |F|^2, the core norm, the
    reconstruction and E against the oracle's."""
    from paper_1711_06874_gb300 import binding

    precision = getattr(binding, precision_name)
    u = U64 if precision == binding.TK_FP64 else U_SLICED
    probs = [wl.problem(wl.MATERN_SD, nu=0.4, p=alpha, n=n, eps=1e-6, rmax=24)
             for alpha, n in ((0.1, 36), (1.0, 32), (100.0, 40))]
    res = ctx.batch(probs, precision=precision, with_error=True)
    for p, r in zip(probs, res):
        ref = orc.hosvd(wl.oracle_kernel(p, orc), wl.oracle_grid(p, orc), p.eps, rmax=list(p.rmax))
        ranks, _ = r.ranks
        if ranks != ref["ranks"]:
            assert any(near_threshold(ref["lam"][a], ref["normF2"], p.eps, ref["ranks"][a]) for a in range(3))
            continue
        nF = math.sqrt(ref["normF2"])
        assert abs(r.norm2 - ref["normF2"]) <= 1e-13 * ref["normF2"]
        assert abs(np.linalg.norm(r.core()) - math.sqrt(ref["core_norm2"])) <= max(1e-12, 100 * u) * nF
        U = [r.factor(a) for a in range(3)]
        X = orc.reconstruct(r.core(), U, p.n)
        Xo = orc.reconstruct(ref["core"], ref["U"], p.n)
        assert np.linalg.norm(X - Xo) <= max(1e-12, 100 * u / p.eps) * nF
        F = orc.tensor(wl.oracle_kernel(p, orc), wl.oracle_grid(p, orc))
        e_or = orc.rel_error(F, X)
        assert abs(r.solve_error - e_or) <= 1e-5 * e_or + 1e-15


def test_sliced_error_above_eps_is_solved_again_in_fp64(ctx, wl):
    """The spectral density at n = 256 (nu = 0.4, alpha = 0.1) is a case where
    the sliced Gram's E (about 1e-6 at rank 11: 0.98e-6 to 1.5e-6 as the start
    block's rounding goes) lands above eps = 5e-7 although the rank rule's sums
    do not, while the FP64 Gram's (3.98e-7) meets it: with with_error the
    instance comes back solved again with the FP64 Gram (flag
    TK_SOLVED_AGAIN_IN_FP64), with E <= eps and the bytes of a plain FP64
    solve.  A Matern instance in the same batch keeps its sliced result."""
    from paper_1711_06874_gb300 import binding

    sd = wl.problem(wl.MATERN_SD, nu=0.4, p=0.1, n=256, eps=5e-7, rmax=24)
    mat = wl.problem(0, nu=1.2, ell=0.2, n=64, eps=1e-6, rmax=24)
    res = ctx.batch([sd, mat], precision=binding.TK_SLICED_BF16, with_error=True)
    r_sd, r_mat = res[0], res[1]
    _, f_sd = r_sd.ranks
    _, f_mat = r_mat.ranks
    assert all(f & binding.TK_SOLVED_AGAIN_IN_FP64 for f in f_sd)
    assert not any(f & binding.TK_SOLVED_AGAIN_IN_FP64 for f in f_mat)
    assert r_sd.solve_error <= sd.eps
    assert r_mat.solve_error <= mat.eps
    ref = ctx.tucker(sd, precision=binding.TK_FP64, with_error=True)
    assert r_sd.ranks[0] == ref.ranks[0]
    assert r_sd.solve_error == ref.solve_error
    for a in range(3):
        assert _same(r_sd.factor(a), ref.factor(a)), a
    assert _same(r_sd.core(), ref.core())
    one = ctx.tucker(sd, precision=binding.TK_SLICED_BF16, with_error=True)
    assert all(f & binding.TK_SOLVED_AGAIN_IN_FP64 for f in one.ranks[1])
    assert one.solve_error <= sd.eps


def test_large_batch_speculation_and_replay_bitwise(ctx, wl):
    """Batches above the small-batch size speculate once a batch of the same
    plan needed no more eigenpairs than the first pass computes, and are then
    captured and replayed as one CUDA graph: every repetition gives the bits
    of the first (plain) run and of each instance alone.  A batch of the same
    plan whose instances need more pairs (eps = 1e-10) makes the speculation
    fail; it is redone the ordinary way and still matches each instance alone."""
    from paper_1711_06874_gb300 import binding

    rng = np.random.default_rng(77)
    probs = [wl.problem(0, nu=float(rng.uniform(0.8, 2.5)), ell=float(rng.uniform(0.3, 0.8)), n=48, eps=1e-5,
                        rmax=24) for _ in range(16)]
    for precision in (binding.TK_SLICED_BF16, binding.TK_FP64):
        args = binding.BatchArgs(probs, precision=precision)
        runs = [ctx.batch(args) for _ in range(4)]  # plain, speculative plain, captured, replayed
        assert max(r.ranks[0][0] for r in runs[0]) <= 12  # the first pass covers every instance
        for rep in runs[1:]:
            for r0, r in zip(runs[0], rep):
                assert r.ranks == r0.ranks and r.norm2 == r0.norm2
                assert _same(r.core(), r0.core())
                for a in range(3):
                    assert _same(r.factor(a), r0.factor(a))
        for p, r in zip(probs[:4], runs[3][:4]):
            alone = ctx.tucker(p, precision=precision)
            assert _same(r.core(), alone.core())
            assert _same(r.factor(0), alone.factor(0))
        # the same plan with instances that need more than the first pass's pairs
        tight = [wl.problem(0, nu=0.5 + 0.02 * i, ell=0.12, n=48, eps=1e-10, rmax=24) for i in range(16)]
        rt = ctx.batch(tight, precision=precision)
        assert max(r.ranks[0][0] for r in rt) > 12
        for p, r in zip(tight[:4], rt[:4]):
            alone = ctx.tucker(p, precision=precision)
            assert r.ranks == alone.ranks
            assert _same(r.core(), alone.core())
            assert _same(r.factor(0), alone.factor(0))
        # and the plan speculates again only after a batch that held
        again = ctx.batch(args)
        for r0, r in zip(runs[0], again):
            assert _same(r.core(), r0.core())
