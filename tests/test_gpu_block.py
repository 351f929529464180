"""Block right-hand sides: nrhs columns through every stage of the solve path
at once (SpMV, restriction, local solves, prolongation, the multifrontal
coarse solve with k columns per tile task, PCG with per-column scalars and
freezing).  Every column's arithmetic is the single-column arithmetic, so a
block result must equal the single-column results bit for bit; the solutions
are also checked against the oracle's direct solve.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def blk():
    import paper_2311_18783_gb300 as pkg
    import workloads as W
    from test_gpu_parity import hetero_box
    import dataclasses
    w = hetero_box(seed=9)
    nverts = (w.nx + 1) * (w.ny + 1) * (w.nz + 1)
    w5 = dataclasses.replace(w, f_slot=W._uniform_f(np.random.default_rng(21), nverts, 5))
    s = pkg.Solver.from_workload(w5, precision=pkg.PREC_FP32, use_graph=1)
    se = pkg.Solver.from_workload(w5, precision=pkg.PREC_FP32, use_graph=0)
    B = torch.empty((5, s.n), dtype=torch.float64, device="cuda")
    for j in range(5):
        s.assemble_rhs(w5.f_slot[j], B[j])
    B[3].zero_()  # a zero right-hand side converges at once
    yield pkg, w5, s, se, B
    s.close()
    se.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_block_apply_equals_columns(blk, prec):
    pkg, w, s, se, B = blk
    s.use_precision(pkg.PREC_FP64 if prec == "fp64" else pkg.PREC_FP32)
    R = torch.as_tensor(np.random.default_rng(2).standard_normal((5, s.n)), device="cuda")
    Z = torch.empty_like(R)
    s.apply_preconditioner_block(R, Z)
    for j in range(5):
        z = torch.empty_like(R[j])
        s.apply_preconditioner(R[j].contiguous(), z)
        assert torch.equal(Z[j], z)


@pytest.mark.parametrize("balanced", [0, 1])
@pytest.mark.parametrize("graph", [1, 0])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_block_solve_equals_columns(blk, prec, graph, balanced):
    pkg, w, s, se, B = blk
    sv = s if graph else se
    sv.use_precision(pkg.PREC_FP64 if prec == "fp64" else pkg.PREC_FP32)
    sv.use_balanced(bool(balanced))
    try:
        X = torch.empty_like(B)
        st, infos = sv.solve_block(B, X, tol=1e-10, maxit=500)
        assert st == 0
        assert infos[3]["iters"] == 0 and torch.count_nonzero(X[3]) == 0
        for j in (0, 1, 2, 4):
            x = torch.zeros_like(B[j])
            info = sv.solve(B[j].contiguous(), x, tol=1e-10, maxit=500)
            assert info["iters"] == infos[j]["iters"] > 2
            assert torch.equal(X[j], x)
    finally:
        sv.use_balanced(False)


def test_block_solve_vs_oracle(blk):
    from oracle.mesh import build_mesh
    from oracle.fem import assemble_A
    from oracle.solver import direct_solve
    pkg, w, s, se, B = blk
    s.use_precision(pkg.PREC_FP64)
    X = torch.empty_like(B)
    st, infos = s.solve_block(B, X, tol=1e-12, maxit=500)
    assert st == 0
    m = build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active)
    A = assemble_A(m, w)
    ev = np.linalg.eigvalsh(A.toarray())
    Bh, Xh = B.cpu().numpy(), X.cpu().numpy()
    for j in (0, 1, 2, 4):
        xs = direct_solve(A, Bh[j])
        err = np.linalg.norm(Xh[j] - xs) / np.linalg.norm(xs)
        assert err <= max(2 * (ev[-1] / ev[0]) * 1e-12, 1e-13)


def test_block_limits(blk):
    pkg, w, s, se, B = blk
    X = torch.empty((17, s.n), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.GeneoError):
        s.solve_block(X, X, tol=1e-8)
