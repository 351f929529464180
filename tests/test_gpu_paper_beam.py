"""The paper's weak-scaling beam (Sec. 4, Table "homogeneous_beam_both"):
(N/2) x 1 x 1 with N = 8 boxes along the length, one overlap layer,
mu = eps = 1, f = (1, 1, 1), gamma = 1e-3, GenEO threshold lambda > 10,
AS-SNK-GenEO, right-preconditioned GMRES to a relative residual of 1e-6 (the
paper's Krylov method and stopping rule), Dirichlet conditions on all faces
or Neumann conditions on the two y faces (mixed).

At h = 1/8 the library is compared with the oracle (dense eigensolves of
every subdomain): GenEO counts per subdomain exactly (0 Dirichlet, as the
paper prints; 1 per interior subdomain with mixed conditions, eigenvalue
near 4e4), the eigenvalues to 1e-6, and the GMRES iteration count (+-1).

At the paper's h = 1/16 (with GENEO_GPU_LONG=1) the oracle's dense eigensolves are out of reach
(eight subdomains of 17,700 unknowns); the library's GenEO sizes and GMRES
counts are printed beside the paper's (0 GenEO vectors; 14 Dirichlet and 15
mixed iterations).  They differ in the GenEO size: with the Boolean
partition of unity the filtered GEVP's top eigenvalue grows like 1/h
(2.7 at h = 1/4, 5.6 at h = 1/8 in the oracle) and crosses tau = 10 at
h = 1/16, so GenEO adds one or two vectors per interior subdomain; the test
checks convergence and an iteration count within 6 of the paper's."""
import numpy as np
import pytest

import workloads as W

from conftest import GPU_LONG

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PAPER = {"dirichlet": 14, "mixed": 15}


def _beam(m, bc):
    w = W.box(4 * m, m, m, h=1 / m, parts=(8, 1, 1), overlap=1, gamma=1e-3, tau=0.1)
    if bc == "mixed":
        w.natural = W.natural_faces(w, sides=((1, 0), (1, 1)))
    return w


@pytest.mark.parametrize("bc", ["dirichlet", "mixed"])
def test_beam_h8_against_oracle(bc):
    import paper_2311_18783_gb300 as pkg
    from oracle.pipeline import build_problem
    from oracle.solver import gmres_right
    w = _beam(8, bc)
    prob = build_problem(w)
    s = pkg.Solver.from_workload(w)
    ref = [int((g.lam > prob.tau_p).sum()) for g in prob.gevps]
    assert list(s.export("geneo_found")) == ref
    assert sum(ref) == (0 if bc == "dirichlet" else 6)
    sub, lam = s.export("geneo_sub"), s.export("geneo_lambda")
    for j, g in enumerate(prob.gevps):
        want = g.lam[g.lam > prob.tau_p]
        for x in lam[sub == j]:
            assert np.abs(want - x).min() <= 1e-6 * want.max()
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(w.f_slot[0], b)
    x = torch.zeros_like(b)
    gi = s.solve_gmres(b, x, tol=1e-6, maxit=300, restart=100)
    ro = gmres_right(prob.A, prob.b[0], prob.M.apply, tol=1e-6, restart=100)
    print(f"h = 1/8 {bc}: GenEO {sum(ref)}, GMRES {gi['iters']} (oracle {ro.iters})")
    assert gi["status"] == 0 and abs(gi["iters"] - ro.iters) <= 1
    s.close()


@pytest.mark.skipif(not GPU_LONG, reason="long GPU test (two set-ups with 17,700-unknown "
                    "subdomains): set GENEO_GPU_LONG=1")
@pytest.mark.parametrize("bc", ["dirichlet", "mixed"])
def test_paper_beam_n8(bc):
    import paper_2311_18783_gb300 as pkg
    w = W.paper_beam(8)
    if bc == "mixed":
        w.natural = W.natural_faces(w, sides=((1, 0), (1, 1)))
    s = pkg.Solver.from_workload(w)
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(w.f_slot[0], b)
    x = torch.zeros_like(b)
    g = s.solve_gmres(b, x, tol=1e-6, maxit=300, restart=100)
    lam = s.export("geneo_lambda")
    print(f"h = 1/16 {bc}: GenEO {s.sizes['n0_geneo']} (paper 0; eigenvalues "
          f"{np.round(np.sort(lam)[::-1][:6], 2).tolist()}), GMRES {g['iters']} iterations "
          f"(paper {PAPER[bc]}), relres {g['relres']:.2e}, n0 {s.sizes['n0']}")
    assert g["status"] == 0 and g["relres"] <= 1e-6
    assert abs(g["iters"] - PAPER[bc]) <= 6
    s.close()
