"""PCG with the iteration captured as a CUDA graph against plain launches.

Every kernel on the solve path is deterministic (fixed-order reductions, no
atomics in the sums), so replaying the captured iteration must give the same
bits as launching it, in float64 and in mixed precision, after switching
precision (the graph is rebuilt), and with profiling on (the graph then
carries event-record nodes around the local and coarse solves).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pair():
    import paper_2311_18783_gb300 as pkg
    from test_gpu_parity import hetero_box
    w = hetero_box(seed=7)
    sg = pkg.Solver.from_workload(w, precision=pkg.PREC_FP32, use_graph=1)
    se = pkg.Solver.from_workload(w, precision=pkg.PREC_FP32, use_graph=0)
    yield pkg, w, sg, se
    sg.close()
    se.close()


def _solve(s, w, tol=1e-10):
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(w.f_slot[0], b)
    x = torch.zeros_like(b)
    info = s.solve(b, x, tol=tol, maxit=500)
    torch.cuda.synchronize()
    return x, info


@pytest.mark.parametrize("prec", ["fp32", "fp64", "fp32_again"])
def test_graph_equals_launches(pair, prec):
    pkg, w, sg, se = pair
    p = pkg.PREC_FP64 if prec == "fp64" else pkg.PREC_FP32
    sg.use_precision(p)
    se.use_precision(p)
    xg, ig = _solve(sg, w)
    xe, ie = _solve(se, w)
    assert ig["status"] == 0 and ie["status"] == 0
    assert ig["iters"] == ie["iters"] and ig["iters"] > 2
    assert torch.equal(xg, xe)
    # a second replay of the cached graph
    xg2, ig2 = _solve(sg, w)
    assert torch.equal(xg2, xg) and ig2["iters"] == ig["iters"]


def test_graph_profiling(pair):
    pkg, w, sg, se = pair
    sg.use_precision(pkg.PREC_FP32)
    se.use_precision(pkg.PREC_FP32)
    out = []
    for s in (sg, se):
        s.profile(True)
        s.profile_read()
        x, info = _solve(s, w)
        prof = s.profile_read()
        s.profile(False)
        out.append((info, prof))
    (ig, pg), (ie, pe) = out
    # one local solve per preconditioner apply: iterations + the initial one
    # (the apply of the converged iteration is not run)
    assert pg["local_symv_launches"] == pe["local_symv_launches"] == ie["iters"]
    assert pg["coarse_symv_launches"] == pe["coarse_symv_launches"] == 2 * ie["iters"]
    # the graph iterates on the context's own x and copies it out once
    assert pg["launches"] == pe["launches"] + 1
    assert pg["local_symv_ms"] > 0 and pe["local_symv_ms"] > 0


def test_bad_option_rejected():
    import paper_2311_18783_gb300 as pkg
    from test_gpu_parity import hetero_box
    with pytest.raises(pkg.GeneoError):
        pkg.Solver.from_workload(hetero_box(seed=7), use_graph=2)
