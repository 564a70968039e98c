"""Writes matern_n512.json: the FP64 oracle's HOSVD (Sec. 3.2) of the n = 512
Matern tensor (nu = 2.5, ell = 0.1, sigma2 = 1, cell-centred grid on
[-1, 1]^3, eps = 1e-6, rank cap 64), which the oracle needs minutes for.

Calls only the oracle.  The grid and the kernel are isotropic, so the three
mode Grams are the same matrix; the script checks that the oracle's three
factors agree and stores mode 1's.  Stored: ranks, flags, |F|^2, |B|^2, E,
the 16 leading eigenvalues, the factor (512 x r) and the core (r x r x r).

    python tests/golden/make_matern_n512.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def main():
    import oracle
    from paper_1711_06874_gb300 import workloads

    oracle.build()
    prob = workloads.matern_n512(1e-6)
    ref = oracle.hosvd(workloads.oracle_kernel(prob, oracle), workloads.oracle_grid(prob, oracle), prob.eps,
                       rmax=list(prob.rmax))
    for a in (1, 2):
        assert ref["ranks"][a] == ref["ranks"][0]
        assert np.array_equal(ref["U"][a], ref["U"][0]), "the isotropic factors should be equal"
        assert np.array_equal(ref["lam"][a][:16], ref["lam"][0][:16])
    out = {
        "source": "oracle.hosvd of workloads.matern_n512(1e-6); Sec. 3.2 HOSVD, Eq. (Matern), Eq. (FNorm)",
        "n": list(prob.n), "nu": prob.nu, "ell": list(prob.ell), "eps": prob.eps, "rmax": list(prob.rmax),
        "ranks": ref["ranks"], "flags": ref["flags"], "normF2": ref["normF2"], "core_norm2": ref["core_norm2"],
        "rel_error": ref["rel_error"], "lam": [float(v) for v in ref["lam"][0][:16]],
        "U": [[float(v) for v in row] for row in ref["U"][0]],
        "core": [float(v) for v in ref["core"].ravel()],
    }
    with open(os.path.join(HERE, "matern_n512.json"), "w") as fh:
        json.dump(out, fh, indent=0)
        fh.write("\n")


if __name__ == "__main__":
    main()
