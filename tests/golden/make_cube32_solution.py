"""Writes tests/golden/cube32_solution.npy from the CPU oracle alone.

Workload: the 32^3 unit cube with the central 8x8x32 hole and four random
2x2 mu^-1 channels (workloads.cube32_hole_channels, seed 2), gamma = 1e-4,
its seeded right-hand side b = l(v) (Sec. 2).

Stored: x = A^-1 b (float64, unknown order) from oracle.solver.
refined_direct_solve: a sparse LU of A followed by three rounds of
iterative refinement with extended-precision residuals.  A plain float64
solve of this system has a forward error near 1e-7 (the float64 residual of
a float64 x cannot fall below u ||A|| ||x||, and gamma = 1e-4 makes the
gradient part of x large); the refinement brings the corrections to about
1e-10 of x.  The refinement history is written beside it as JSON, with the
solution's sensitivity to its own float64 data: the same refined solve with
every stored entry of A multiplied by 1 +- 2^-53 (random signs, symmetric),
i.e. a one-ulp change, moves x by `one_ulp_sensitivity` (relative).  Two
independent float64 assemblies of A differ by that much, so no solution of
an independently assembled system can agree with this one more closely.

Run from the repository root: python tests/golden/make_cube32_solution.py
(about eight minutes, most of it the two sparse LU factorisations).
"""
import json
import os
import sys
import time

import numpy as np
import scipy.sparse as sp

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle.mesh import build_mesh  # noqa: E402
from oracle.fem import assemble_A, assemble_rhs  # noqa: E402
from oracle.solver import refined_direct_solve, residual_extended  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    t0 = time.time()
    w = W.cube32_hole_channels()
    m = build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active)
    A = assemble_A(m, w)
    b = assemble_rhs(m, w)[0]
    x, hist = refined_direct_solve(A, b, steps=3)
    res = residual_extended(A, b, x).astype(np.float64)
    np.save(os.path.join(HERE, "cube32_solution.npy"), x)
    rng = np.random.default_rng(0)
    U = sp.triu(A, format="coo")
    d = U.data * (1.0 + 2.0 ** -53 * rng.choice([-1.0, 1.0], U.data.shape))
    Up = sp.coo_matrix((d, (U.row, U.col)), shape=A.shape)
    xp, _ = refined_direct_solve((Up + sp.triu(Up, 1).T).tocsr(), b, steps=3)
    sens = float(np.linalg.norm(xp - x) / np.linalg.norm(x))
    meta = {"workload": "cube32_hole_channels", "n": int(A.shape[0]),
            "method": "sparse LU + 3 rounds of refinement with longdouble residuals",
            "correction_rel_sizes": hist,
            "extended_relres": float(np.linalg.norm(res) / np.linalg.norm(b)),
            "longdouble_significand_bits": int(np.finfo(np.longdouble).nmant) + 1,
            "one_ulp_sensitivity": sens,
            "seconds": time.time() - t0}
    with open(os.path.join(HERE, "cube32_solution.json"), "w") as f:
        json.dump(meta, f, indent=1)
    print(meta)


if __name__ == "__main__":
    main()
