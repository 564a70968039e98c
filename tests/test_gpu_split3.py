"""The BF16x3 and TF32x3 Gram variants (TK_BF16X3, TK_TF32X3) through the C-ABI.

Each entry is rounded to FP32 and split into two BF16 (or TF32) terms; the
tensor cores sum the three products hi hi + hi lo + lo hi in FP32.

  * Gram, small integers: every term and every partial sum is exact in these
    formats, so G equals the integer Gram exactly (a layout, descriptor or
    index mistake in the kernel cannot pass);
  * Gram, real data against the oracle: per entry within the rounding bound
    (c u + 2 K 2^-24) (|A| |A|^T)_ij of the split and the FP32 sums, and within
    2^-14 max|G| overall;
  * whole solve against the oracle at eps = 1e-4, 1e-6 and 1e-8: factors
    orthonormal, the core the FP64 TTM chain of the returned factors, E of
    the returned factors equal to the oracle's E of the same factors, the
    unreachable-eps flag set exactly where eps^2 / 3 < 10 u n, and the
    measured E against the oracle's E, recorded.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# unit roundoff of each variant's Gram as the library states it (rank rule flag)
U_VAR = {"TK_BF16X3": 2.0 ** -16, "TK_TF32X3": 2.0 ** -21}


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


@pytest.mark.parametrize("precision_name", ["TK_BF16X3", "TK_TF32X3"])
@pytest.mark.parametrize("shape", [(96, 40, 50), (200, 3, 5), (2, 2, 2), (130, 9, 40)])
def test_gram_split3_exact_on_small_integers(ctx, precision_name, shape):
    """|x| <= 15: hi = x, lo = 0, and every partial sum stays below 2^24."""
    from paper_1711_06874_gb300 import binding

    rng = np.random.default_rng(31)
    Fh = rng.integers(-15, 16, size=shape).astype(np.float64)
    F = _dev(Fh)
    for mode in range(3):
        A = np.moveaxis(Fh, mode, 0).reshape(shape[mode], -1).astype(np.int64)
        exact = (A @ A.T).astype(np.float64)
        G = torch.full(exact.shape, float("nan"), dtype=torch.float64, device="cuda")
        ctx.gram(F, mode, G, precision=getattr(binding, precision_name))
        np.testing.assert_array_equal(G.cpu().numpy(), exact)


@pytest.mark.parametrize("precision_name", ["TK_BF16X3", "TK_TF32X3"])
@pytest.mark.parametrize("shape", [(70, 45, 33), (64, 64, 64), (256, 16, 16), (5, 130, 9)])
def test_gram_split3_matches_oracle(ctx, orc, precision_name, shape):
    from paper_1711_06874_gb300 import binding

    rng = np.random.default_rng(23)
    Fh = rng.random(shape) * np.exp(-3 * rng.random(shape))
    F = _dev(Fh)
    u = U_VAR[precision_name]
    for mode in range(3):
        m = shape[mode]
        G = torch.empty((m, m), dtype=torch.float64, device="cuda")
        ctx.gram(F, mode, G, precision=getattr(binding, precision_name))
        ref = orc.gram(Fh, mode)
        got = G.cpu().numpy()
        A = np.abs(np.moveaxis(Fh, mode, 0).reshape(m, -1))
        K = A.shape[1]
        # per product: FP32 input rounding, the split's residual and the dropped
        # lo lo term (< 4 u); the FP32 sums over at most K terms (2 K 2^-24)
        bound = (4 * u + 2 * K * 2.0 ** -24) * (A @ A.T)
        assert (np.abs(got - ref) <= bound).all(), (shape, mode, np.abs(got - ref).max())
        assert np.abs(got - ref).max() <= 2.0 ** -14 * np.abs(ref).max(), (shape, mode)


@pytest.mark.parametrize("precision_name", ["TK_BF16X3", "TK_TF32X3"])
@pytest.mark.parametrize("n", [64, 256])
def test_tucker_split3_error_against_oracle(ctx, orc, wl, precision_name, n):
    from paper_1711_06874_gb300 import binding

    precision = getattr(binding, precision_name)
    u = U_VAR[precision_name]
    for eps in (1e-4, 1e-6, 1e-8):
        prob = wl.slater_n64(eps) if n == 64 else wl.matern_n256(eps)
        kern, grid = wl.oracle_kernel(prob, orc), wl.oracle_grid(prob, orc)
        ref = orc.hosvd(kern, grid, prob.eps, rmax=list(prob.rmax))
        res = ctx.tucker(prob, precision=precision)
        ranks, flags = res.ranks
        U = [res.factor(a) for a in range(3)]
        B = res.core()
        for a in range(3):
            np.testing.assert_allclose(U[a].T @ U[a], np.eye(ranks[a]), atol=1e-13)
            want = (eps * eps / 3.0) < 10.0 * u * prob.n[a]
            assert bool(flags[a] & binding.TK_EPS_UNREACHABLE_AT_PRECISION) == want, (a, flags)
        F = orc.tensor(kern, grid)
        nF = math.sqrt(ref["normF2"])
        # the core is the FP64 TTM chain of the returned factors
        np.testing.assert_allclose(B, orc.core(F, U, ranks), rtol=0, atol=1e-12 * nF)
        e = res.rel_error()
        e_own = orc.rel_error(F, orc.reconstruct(B, U, prob.n))
        assert abs(e - e_own) <= 1e-10 * e_own + 1e-15
        print(f"{precision_name} n={n} eps={eps:g}: ranks {ranks} E {e:.4e} oracle E {ref['rel_error']:.4e} "
              f"ratio {e / ref['rel_error']:.3g}")
        res.free()
