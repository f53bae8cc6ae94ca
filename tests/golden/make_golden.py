"""Write the oracle-derived expected values of tests/golden/.

The thesis's one small worked example (Ch. 2, Ex. "nonconverging_gmres") is
stored by hand in gmres_cyclic_shift.json with its citation; its numeric tables
are measured on SuiteSparse matrices with SSOR / ILU preconditioners, so the
other stored values are the oracle's own, written by this
script, which imports nothing but ``oracle`` and ``workloads``:

  bcg_poisson2d_12x11_s3.json  Alg. "bcgaro" (Ch. 4.3), 12 x 11 Dirichlet Poisson
                               (5-point, unscaled), s = 3, B seed 0: per-iteration
                               max-column relative residuals, decisions and kappa_D
                               for eta = inf, 0 and 1e4; Alg. "1R-CG" (Ch. 8.1) for
                               eta = inf; point Jacobi on a log-normal 5^3 FV field.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "..", ".."))
import oracle  # noqa: E402
import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _run(fn, A, B, **kw):
    r = fn(A, B, tol=1e-10, maxit=500, **kw)
    return {"iters": r.iters, "reorths": r.reorths, "converged": r.converged,
            "history": [float(h) for h in r.history],
            "decisions": [bool(d) for d in r.decisions],
            "kappas": [None if k is None else float(k) for k in r.kappas],
            "X_first_row": [float(v) for v in r.X[0]]}


def main():
    A = W.lap2d5(12, 11)
    B = W.normal_block(A.n, 3, 0)
    k = np.exp(1.5 * np.random.default_rng(5).standard_normal(125))
    Av = W.diff3d7_var(5, 5, 5, k)
    Bv = W.normal_block(Av.n, 3, 1)
    out = {
        "source": "oracle (tests/golden/make_golden.py); Alg. bcgaro (Ch. 4.3), Alg. 1R-CG (Ch. 8.1)",
        "problem": "poisson2d 12x11 5-point Dirichlet, s=3, B = normal_block(n, 3, seed 0); "
                   "vardiff 5^3 k = exp(1.5 g), g seed 5, s=3, B seed 1",
        "bcg_eta_inf": _run(oracle.bcg, A, B, eta=math.inf),
        "bcg_eta_0": _run(oracle.bcg, A, B, eta=0.0),
        "bcg_eta_1e4": _run(oracle.bcg, A, B, eta=1e4),
        "bcg_1r_eta_inf": _run(oracle.bcg_1r, A, B, eta=math.inf),
        "bcg_jacobi_vardiff_eta_inf": _run(oracle.bcg, Av, Bv, eta=math.inf,
                                           Minv=oracle.jacobi_inverse_diagonal(Av)),
    }
    with open(os.path.join(HERE, "bcg_poisson2d_12x11_s3.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
