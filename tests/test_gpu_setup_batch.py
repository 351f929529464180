"""geneo_setup_batch against the same problems composed in Python
(workloads.compose).  The library's composition equals the Python one bit
for bit (test_capi_compose.py), so the two contexts must give the same
unknowns and the same segmented solution bit for bit.  Collected after the
rest of the GPU suite."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    import paper_2311_18783_gb300 as pkg
    from test_gpu_batch import _problems
    ps = _problems()
    c = W.compose(ps)
    s = pkg.Solver.from_workload(c)
    yield pkg, ps, c, s
    s.close()


def test_setup_batch_equals_composed_problem(batch):
    pkg, ps, c, s = batch
    sb = pkg.Solver.batch(ps)
    assert sb.n == s.n and sb.sizes["n0"] == s.sizes["n0"]
    assert np.array_equal(sb.export("seg_off"), s.export("seg_off"))
    f = pkg.compose(ps)["f_slot"]
    assert np.array_equal(f, c.f_slot)
    b1 = torch.empty(s.n, dtype=torch.float64, device="cuda")
    b2 = torch.empty_like(b1)
    s.assemble_rhs(c.f_slot[0], b1)
    sb.assemble_rhs(f[0], b2)
    x1, x2 = torch.zeros_like(b1), torch.zeros_like(b1)
    st1, i1 = s.solve_segments(b1, x1, tol=1e-10, maxit=500)
    st2, i2 = sb.solve_segments(b2, x2, tol=1e-10, maxit=500)
    assert st1 == st2 == 0
    assert [d["iters"] for d in i1] == [d["iters"] for d in i2]
    assert torch.equal(x1, x2)
    sb.close()
