"""Serving loop (tk_serve_start / tk_submit / tk_poll) on the GPU.

  * every result of a concurrent mix is checked against the FP64 oracle's
    HOSVD of that request (ranks, |F|^2, core norm, reconstruction, principal
    angles, E; the small cases' tolerances) and is bitwise the one tk_tucker
    returns for that request alone, and requests were in fact batched
    together; a second mix includes n = 128 requests;
  * a short Poisson stream replayed in real time completes with positive
    latencies;
  * argument and state errors come back as status codes.
"""
import time

import numpy as np
import pytest

from tests._util import U64, compare_solution

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture()
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


U_SLICED = 2.0 ** -48


def _mix(wl, count=40, seed=5, sizes=(32, 48, 64)):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        nu = float(rng.uniform(0.3, 2.5))
        ell = float(np.exp(rng.uniform(np.log(0.05), 0.0)))
        eps = float(rng.choice([1e-4, 1e-6, 1e-8]))
        out.append(wl.problem(0, nu=nu, ell=ell, n=n, eps=eps, rmax=24))
    return out


@pytest.mark.parametrize("precision_name", ["TK_SLICED_BF16", "TK_FP64"])
@pytest.mark.parametrize("mix", ["small", "with_n128"])
def test_serve_mix_matches_oracle_and_alone(ctx, orc, wl, precision_name, mix):
    from paper_1711_06874_gb300 import binding

    precision = getattr(binding, precision_name)
    u = U64 if precision == binding.TK_FP64 else U_SLICED
    probs = _mix(wl) if mix == "small" else _mix(wl, count=12, seed=11, sizes=(64, 128))
    ctx.serve_start(workers=2, max_batch=64)
    tickets = [ctx.submit(p, precision=precision) for p in probs]
    got = []
    for t in tickets:
        r = ctx.poll(t, wait_s=60.0)
        assert r is not None
        got.append(r)
    stats = ctx.serve_stats()
    ctx.serve_stop()
    assert stats["completed"] == len(probs) and stats["failed"] == 0
    assert stats["max_batch_seen"] > 1 and stats["batches"] < len(probs)
    for p, (res, lat) in zip(probs, got):
        assert lat > 0.0
        ref, e = compare_solution(orc, wl, res, p, precision_u=u)
        if precision != binding.TK_FP64:
            # the sliced Gram's E against the oracle's (unless flagged below its precision)
            assert e <= 2 * ref["rel_error"] or any(res.ranks[1]), (p, e, ref["rel_error"])
        alone = ctx.tucker(p, precision=precision)
        assert res.ranks == alone.ranks
        assert res.norm2 == alone.norm2
        assert np.array_equal(res.core(), alone.core())
        for a in range(3):
            assert np.array_equal(res.factor(a), alone.factor(a))
        alone.free()
        res.free()


def test_serve_poisson_stream_small(ctx, wl):
    from paper_1711_06874_gb300 import binding

    stream = wl.serving_stream(count=80, rate_hz=400.0)
    ctx.serve_start(workers=2)
    t0 = time.perf_counter()
    tickets = []
    for at, p in stream:
        p = wl.problem(0, nu=p.nu, ell=p.ell[0], n=min(p.n[0], 128), eps=p.eps, rmax=p.rmax[0])
        delay = at - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        tickets.append(ctx.submit(p, precision=binding.TK_SLICED_BF16))
    lats = []
    for t in tickets:
        r = ctx.poll(t, wait_s=120.0)
        assert r is not None
        res, lat = r
        assert res.ranks[0][0] >= 1
        lats.append(lat)
        res.free()
    stats = ctx.serve_stats()
    ctx.serve_stop()
    assert stats["completed"] == len(stream)
    assert min(lats) > 0 and np.percentile(lats, 99) < 60.0


def test_serve_errors(ctx, wl):
    from paper_1711_06874_gb300 import binding

    lib = binding.load()
    import ctypes

    out = ctypes.c_void_p()
    # not serving yet
    assert lib.tk_poll(ctx.ptr, 1, ctypes.byref(out), None, 0.0) == binding.TK_EINVAL
    ctx.serve_start(workers=1)
    with pytest.raises(binding.TuckerError):
        ctx.serve_start(workers=1)  # already serving
    assert lib.tk_poll(ctx.ptr, 12345, ctypes.byref(out), None, 0.0) == binding.TK_ENOTFOUND
    with pytest.raises(binding.TuckerError) as ei:
        ctx.submit(wl.problem(0, nu=-1.0, n=16))
    assert ei.value.status == binding.TK_EINVAL
    with pytest.raises(binding.TuckerError) as ei:
        ctx.submit(wl.problem(0, nu=1.0, n=16, rmax=12), rfix=(12, 12, 12))  # above the even vectors
    assert ei.value.status == binding.TK_EINVAL
    t = ctx.submit(wl.problem(0, nu=1.0, ell=0.3, n=16, rmax=8))
    res, _ = ctx.poll(t, wait_s=30.0)
    assert res.ranks[0][0] >= 1
    assert lib.tk_poll(ctx.ptr, t, ctypes.byref(out), None, 0.0) == binding.TK_ENOTFOUND  # taken
    ctx.serve_stop()
    with pytest.raises(binding.TuckerError):
        ctx.serve_stop()
