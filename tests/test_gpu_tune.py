"""Autotuning of the sliced Gram's K split (tk_tune) on the GPU.

The sliced Gram sums exact integer chunks, so its result does not depend on
how K is split: with tuning on, every Gram and every whole solve is bitwise
the untuned one; the choices are written to the JSON cache and read back.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture()
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_06874_gb300 import binding

    c = binding.Context(0)
    yield c
    c.tune(False, "")  # tuning is process-wide: leave it off for the other tests
    c.close()


def test_tuned_gram_and_solve_are_bitwise_the_default(ctx, tmp_path):
    from paper_1711_06874_gb300 import binding, workloads

    rng = np.random.default_rng(4)
    shapes = [(64, 64, 64), (128, 96, 80), (40, 33, 70)]
    tensors = [torch.from_numpy(rng.random(sh) * np.exp(-3 * rng.random(sh))).cuda() for sh in shapes]
    prob = workloads.problem(0, nu=1.2, ell=0.2, n=128, eps=1e-6, rmax=24)

    def run():
        out = []
        for F, sh in zip(tensors, shapes):
            for mode in range(3):
                G = torch.empty((sh[mode], sh[mode]), dtype=torch.float64, device="cuda")
                ctx.gram(F, mode, G, precision=binding.TK_SLICED_BF16)
                out.append(G.cpu().numpy())
        res = ctx.tucker(prob, precision=binding.TK_SLICED_BF16)
        out.append(res.core())
        out.append(res.factor(0))
        res.free()
        return out

    ctx.tune(False, "")
    base = run()
    path = str(tmp_path / "tune.json")
    ctx.tune(True, path)
    tuned = run()  # first use of each shape: timed candidates, then the choice
    again = run()  # the stored choices
    for a, b, c in zip(base, tuned, again):
        assert a.shape == b.shape and np.array_equal(a, b) and np.array_equal(a, c)
    entries = ctx.tune(True, None)
    assert entries >= 1
    with open(path) as fh:
        stored = json.load(fh)
    assert len(stored) == entries and all(isinstance(v, int) and v >= 1 for v in stored.values())
    # a fresh process state reads the file back: same choices
    ctx.tune(True, path)
    assert ctx.tune(True, None) == entries
    assert os.path.getsize(path) > 2
