"""The tensor-core first TTM of the sliced path at the larger padded ranks.

The core B = Fh x_1 V1^T x_2 V2^T x_3 V3^T of a sliced solve is compared with
the oracle's direct FP64 TTMs of the full tensor on the GPU's own factors,
so that only the core's arithmetic is under test.  Fixed ranks 40 and 70 pad
to Np = 64 (six accumulators side by side, one MMA per A slice over its B
slices, two where N passes 256) and Np = 96 (five accumulators, one MMA per
slice pair).  Bound: the slices carry Fh and V3 to 2^-48 of their row and
column scales, so |B - B_or| stays near 2^-48 h |F|_max per entry; a slice
pair sent to the wrong accumulator moves B by about 2^-8 of a term.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("n,r", [(96, 40), (160, 70)])
def test_sliced_core_at_large_fixed_ranks(ctx, orc, n, r):
    from paper_1711_06874_gb300 import binding, workloads as wl

    prob = wl.problem(0, nu=0.8, ell=0.3, n=n, eps=1e-6, rmax=r)
    res = ctx.tucker(prob, precision=binding.TK_SLICED_BF16, rfix=(r, r, r))
    ranks, _ = res.ranks
    assert ranks == [r, r, r]
    U = [res.factor(a) for a in range(3)]
    F = orc.tensor(wl.oracle_kernel(prob, orc), wl.oracle_grid(prob, orc))
    B_or = orc.core(F, U, (r, r, r))
    B = res.core()
    dev = float(np.abs(B - B_or).max())
    tol = 2.0 ** -44 * (n // 2) * float(np.abs(F).max())
    assert dev <= tol, (dev, tol)
    # the core carries |F|^2 up to the discarded tail (all but rounding here)
    assert abs(float((B ** 2).sum()) - float((F ** 2).sum())) <= 1e-6 * float((F ** 2).sum())
