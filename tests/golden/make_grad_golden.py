"""Write tests/golden/grad_32x32x16.json: the exact optimum of the
differentiation workload's operator on the 32x32x16 grid (control box [-1, 1])
and the gradient of its optimal value, from the FP64 oracle only.

    python tests/golden/make_grad_golden.py

Contents: J*, dJ*/d(d+, d-, e+, e-) (envelope theorem, oracle
objective_gradient), the KKT violation of the oracle's solution, and 64 seeded
sample points of y*, u*, p* (adjoint from the dense solve of B^T p = -J1 (y*-ybar))
and dJ*/dybar.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import fde_inputs as fi  # noqa: E402
import oracle as O  # noqa: E402


def main():
    inst = fi.config_grad_small()
    sol = O.active_set_solve(inst)
    viol = O.kkt_violation(inst, sol)
    grad = O.objective_gradient(inst, sol)
    padj = O.dense_adjoint(inst, sol)
    N = inst.params.N
    idx = sorted(set(int(i) for i in (fi.uniform01(4242, 64) * N).astype(np.int64)))
    out = {
        "source": "oracle.active_set_solve + objective_gradient + dense_adjoint on fde_inputs.config_grad_small()",
        "J": sol.J,
        "dcoef": [grad["dp"], grad["dm"], grad["ep"], grad["em"]],
        "kkt_violation": {k: float(v) for k, v in viol.items()},
        "adjoint_vs_kkt_p_maxabs": float(np.max(np.abs(padj - sol.p))),
        "index": idx,
        "y": [float(sol.y.flat[i]) for i in idx],
        "u": [float(sol.u.flat[i]) for i in idx],
        "p": [float(padj.flat[i]) for i in idx],
        "dJ_dybar": [float(grad["ybar"].flat[i]) for i in idx],
        "y_maxabs": float(np.max(np.abs(sol.y))),
        "p_maxabs": float(np.max(np.abs(padj))),
    }
    with open(os.path.join(HERE, "grad_32x32x16.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
