"""Natural (Neumann) boundary faces on the GPU (Sec. 4, mixed boundary
conditions), against the oracle.  The integer set-up with natural faces is
checked bit for bit on the CPU (test_capi_topology.py); here the whole
path runs on the beam with holes of workloads.beam_holes (4 boxes,
h = 1/8):
* natural hole surfaces: GenEO finds, per box, the oracle's number of
  eigenvalues above tau (3, 5, 5, 3), the coarse space keeps them all, and
  PCG reaches the direct solution within kappa * tol in the oracle's
  iteration count (+-1);
* Dirichlet hole surfaces: GenEO finds nothing (Sec. 4, table
  "beam_holes_both", top), and PCG agrees with the direct solve.
Collected after the rest of the GPU suite."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("natural", [True, False])
def test_beam_holes_against_oracle(natural):
    import paper_2311_18783_gb300 as pkg
    from oracle.pipeline import build_problem
    from oracle.solver import direct_solve, pcg
    w = W.beam_holes(4, natural_holes=natural)
    prob = build_problem(w)
    ref = [int((g.lam > prob.tau_p).sum()) for g in prob.gevps]
    s = pkg.Solver.from_workload(w)
    assert s.n == prob.A.shape[0]
    got = [int(v) for v in s.export("geneo_found")]
    assert got == ref
    assert s.sizes["n0"] == prob.Z.shape[1]
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(w.f_slot[0], b)
    assert np.abs(b.cpu().numpy() - prob.b[0]).max() <= 1e-14 * np.abs(prob.b[0]).max()
    x = torch.zeros_like(b)
    tol = 1e-10
    info = s.solve(b, x, tol=tol, maxit=500)
    assert info["status"] == 0
    xs = direct_solve(prob.A, prob.b[0])
    ev = np.linalg.eigvalsh(prob.A.toarray())
    err = np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs)
    assert err <= max(2 * ev[-1] / ev[0] * tol, 1e-13)
    ro = pcg(prob.A, prob.b[0], prob.M.apply, tol=tol, maxit=500)
    print(f"natural={natural}: GenEO {got}, n0 {s.sizes['n0']}, PCG {info['iters']} "
          f"(oracle {ro.iters})")
    assert abs(ro.iters - info["iters"]) <= 1
    s.close()
