"""Writes tests/golden/cube32_reference.json from the CPU oracle alone.

Workload: the 32^3 unit cube with the central 8x8x32 hole and four random
2x2 mu^-1 channels (workloads.cube32_hole_channels, seed 2), gamma = 1e-4,
4x4x4 boxes, overlap 2, tau = 0.1 read reciprocally (lambda > 10).

Recorded (all computed by oracle/ only):
* per subdomain, the eigenvalues of the filtered GEVP (Sec. 3.2, GEVP
  "tauthresholdAS", eq. "eigAtildeBAS") above the threshold and the largest
  eigenvalue, from a dense generalised eigensolve;
* the split near-kernel column count, the GenEO columns kept (Z full rank,
  eq. "V0GenEOAS"), n0;
* the oracle PCG iteration count and final relative residual to 1e-8 for
  the seeded right-hand side.

Run from the repository root: python tests/golden/make_cube32_reference.py
(about an hour on 8 cores; per-subdomain results are cached in /tmp).
"""
import json
import os
import pickle
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle.mesh import build_mesh  # noqa: E402
from oracle.fem import assemble_A, assemble_rhs, local_element_A  # noqa: E402
from oracle.dd import decompose  # noqa: E402
from oracle.coarse import (snk_columns, local_gevp, assemble_Z, coarse_matrix,  # noqa: E402
                           independent_geneo, tau_paper)
from oracle.solver import build_preconditioner, pcg  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cube32_reference.json")
CACHE = "/tmp/cube32_gevp_cache"


def main():
    os.makedirs(CACHE, exist_ok=True)
    w = W.cube32_hole_channels()
    t0 = time.time()
    mesh = build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active)
    A = assemble_A(mesh, w)
    AT = local_element_A(mesh, w)
    b = assemble_rhs(mesh, w)[0]
    dec = decompose(mesh, w.parts, w.overlap)
    snk = snk_columns(mesh, dec)
    tp = tau_paper(w.tau, "reciprocal")
    per_sub, gcols = [], []
    for j in range(dec.nsub):
        path = os.path.join(CACHE, f"sub{j}.pkl")
        if os.path.exists(path):
            with open(path, "rb") as f:
                rec = pickle.load(f)
        else:
            g = local_gevp(mesh, w, A, AT, dec, j)
            sel = np.nonzero(g.lam > tp)[0]
            Ixi = np.eye(len(g.Ai)) - g.xi
            vecs = [dec.D[j] * (Ixi @ g.V[:, k]) for k in sel.tolist()]
            rec = {"lam_sel": g.lam[sel].tolist(), "lam_max": float(g.lam[0]),
                   "lam_top": g.lam[:16].tolist(), "vecs": vecs}
            with open(path, "wb") as f:
                pickle.dump(rec, f)
            del g
        per_sub.append(rec)
        for v in rec["vecs"]:
            gcols.append((j, 0, dec.N[j].copy(), v))
        print(f"sub {j}: n_j={len(dec.N[j])} found={len(rec['lam_sel'])} "
              f"lam_max={rec['lam_max']:.4g} t={time.time() - t0:.0f}s", flush=True)
    n = A.shape[0]
    E = coarse_matrix(mesh, w, assemble_Z(n, snk + gcols))
    keep = independent_geneo(E, len(snk))
    sel = np.concatenate([np.arange(len(snk)), len(snk) + keep])
    Ek = E.tocsr()[sel][:, sel] if hasattr(E, "tocsr") else E[np.ix_(sel, sel)]
    Z = assemble_Z(n, snk + [gcols[k] for k in keep.tolist()])
    M = build_preconditioner(A, dec, Z, E=Ek)
    t1 = time.time()
    res = pcg(A, b, M.apply, tol=1e-8, maxit=1000)
    t_pcg = time.time() - t1
    out = {
        "workload": w.name,
        "source": "oracle/ (dense generalised eigensolve per subdomain; PCG with the "
                  "literal two-level preconditioner of Sec. 2, eq. AS2)",
        "n": int(n), "nsub": int(dec.nsub), "tau_paper": tp,
        "n0_snk": len(snk), "geneo_found": [len(r["lam_sel"]) for r in per_sub],
        "geneo_kept": int(len(keep)), "n0": int(len(snk) + len(keep)),
        "lam_selected": [r["lam_sel"] for r in per_sub],
        "lam_max": [r["lam_max"] for r in per_sub],
        "lam_top16": [r["lam_top"] for r in per_sub],
        "pcg_tol": 1e-8, "pcg_iters": int(res.iters), "pcg_relres": float(res.relres),
        "oracle_pcg_seconds_here": t_pcg,
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT, "iters", res.iters, flush=True)


if __name__ == "__main__":
    main()
