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
1e-10 of x.  The refinement history is written beside it as JSON.

Run from the repository root: python tests/golden/make_cube32_solution.py
(about five minutes, most of it the sparse LU).
"""
import json
import os
import sys
import time

import numpy as np

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
    meta = {"workload": "cube32_hole_channels", "n": int(A.shape[0]),
            "method": "sparse LU + 3 rounds of refinement with longdouble residuals",
            "correction_rel_sizes": hist,
            "extended_relres": float(np.linalg.norm(res) / np.linalg.norm(b)),
            "longdouble_significand_bits": int(np.finfo(np.longdouble).nmant) + 1,
            "seconds": time.time() - t0}
    with open(os.path.join(HERE, "cube32_solution.json"), "w") as f:
        json.dump(meta, f, indent=1)
    print(meta)


if __name__ == "__main__":
    main()
