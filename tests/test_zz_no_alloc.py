"""Allocation-free Gram entry point, tk_gram_noalloc.

Some callers cannot allocate device memory (a host application whose own
allocator already holds the GPU's memory, real-time loops that must not pay
cudaMalloc's latency or implicit synchronisation, plugins handed only
pointers).  tk_gram_noalloc serves them: it keeps its split-K partial sums in
a fixed device array inside the library.  This test calls it through the
C-ABI twice in a row, on different inputs, and checks each result against
tk_gram (precision TK_FP64) within the Gram tolerance of the parity tests,
1e-13 max|G|.  The 256^3 tensor is large enough that the default K split's
partial sums would not fit the fixed array, so the entry point takes fewer,
longer splits there (its summation order then differs from tk_gram's).  It
then rejects an out-of-range size.  The file's name makes
pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_gram_matches_tk_gram_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_06874_gb300 import binding

    lib = binding.load()
    torch.cuda.set_device(0)
    ctx = binding.Context(0)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(2024)
    # different shapes back to back; none may see an earlier call's partial sums.
    # (256, 256, 256) takes the longer-split branch in every mode.
    for shape in [(70, 45, 33), (130, 9, 64), (256, 256, 256), (40, 20, 30)]:
        F = torch.from_numpy(rng.random(shape)).cuda()
        n = (ctypes.c_int32 * 3)(*shape)
        for mode in range(3):
            m = shape[mode]
            G_ref = torch.empty((m, m), dtype=torch.float64, device="cuda")
            ctx.gram(F, mode, G_ref)
            G = torch.full((m, m), float("nan"), dtype=torch.float64, device="cuda")
            rc = lib.tk_gram_noalloc(F.data_ptr(), n, mode, G.data_ptr(), stream)
            assert rc == binding.TK_OK
            torch.cuda.synchronize()
            ref = G_ref.cpu().numpy()
            got = G.cpu().numpy()
            assert np.isfinite(got).all()
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), (shape, mode)
    # sizes beyond the maximum are rejected
    F = torch.zeros(8, dtype=torch.float64, device="cuda")
    G = torch.zeros(8, dtype=torch.float64, device="cuda")
    bad = (ctypes.c_int32 * 3)(2048, 2, 2)
    assert lib.tk_gram_noalloc(F.data_ptr(), bad, 0, G.data_ptr(), stream) == binding.TK_EINVAL
    ctx.close()
