"""The coarse-space variants of Sec. 4 (AS, AS-SNK, AS-NK, AS-NK-GenEO)
against the oracle's literal preconditioners on the beam with Neumann hole
surfaces (workloads.beam_holes, 4 boxes, h = 1/8), where they differ: PCG
to 1e-10 reaches the direct solution within kappa * tol, in the oracle's
iteration count (+-1), with the oracle's coarse dimension.  The NK columns
themselves are checked bit for bit on the CPU (test_capi_topology.py).
Collected after the rest of the GPU suite."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VARIANTS = {  # name: (library coarse mode, geneo, oracle coarse)
    "AS": (0, 0, "none"),
    "AS-SNK": (1, 0, "snk"),
    "AS-NK": (2, 0, "nk"),
    "AS-NK-GenEO": (2, 1, "nk"),
}


@pytest.fixture(scope="module")
def beam():
    from oracle.solver import direct_solve
    w = W.beam_holes(4)
    from oracle.pipeline import build_problem
    p0 = build_problem(w, geneo=False, coarse="none")
    xs = direct_solve(p0.A, p0.b[0])
    ev = np.linalg.eigvalsh(p0.A.toarray())
    return w, xs, ev[-1] / ev[0]


@pytest.mark.parametrize("name", sorted(VARIANTS))
def test_variant_against_oracle(beam, name):
    import paper_2311_18783_gb300 as pkg
    from oracle.pipeline import build_problem
    from oracle.solver import pcg
    w, xs, kappa = beam
    mode, geneo, ocoarse = VARIANTS[name]
    prob = build_problem(w, geneo=bool(geneo), coarse=ocoarse)
    s = pkg.Solver.from_workload(w, coarse=mode, geneo=geneo)
    n0 = 0 if prob.Z is None else prob.Z.shape[1]
    assert s.sizes["n0"] == n0
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(w.f_slot[0], b)
    x = torch.zeros_like(b)
    tol = 1e-10
    info = s.solve(b, x, tol=tol, maxit=1000)
    assert info["status"] == 0
    err = np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs)
    assert err <= max(2 * kappa * tol, 1e-13)
    ro = pcg(prob.A, prob.b[0], prob.M.apply, tol=tol, maxit=1000)
    print(f"{name}: n0 {n0}, PCG {info['iters']} (oracle {ro.iters})")
    assert abs(ro.iters - info["iters"]) <= 1
    s.close()
