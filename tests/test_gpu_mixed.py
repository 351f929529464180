"""Mixed precision: float32 local factors inside the float64 PCG.

The local inverse is split as A_j^-1 = G_j S_j^-1 G_j^T + (I - xi_j) A_j^-1
(Sec. 2, eq. "inverseBw"): the gradient part (large, order 1/gamma) stays in
float64, the rest is stored in float32.  Checked against the oracle's local
solves (relative 1e-5: float32 storage of C_j, float32 accumulation) and by
PCG reaching the float64 solution with the float64 iteration count (+-2).
A plain float32 cast of A_j^-1 would lose the non-gradient part entirely for
small gamma; the test on gamma = 1e-5 covers that regime.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cases():
    from test_gpu_parity import hetero_box
    return {
        "cube8": W.unit_cube_8(),
        "hetero_hole": hetero_box(),
        "beam_small_gamma": hetero_box(seed=3, gamma=1e-5, parts=(3, 1, 1), n=(12, 4, 4),
                                       holes=(((5, 7), (1, 3), (0, 4)),)),
    }


CASES = _cases()


@pytest.fixture(scope="module", params=sorted(CASES))
def mcase(request):
    import paper_2311_18783_gb300 as pkg
    from oracle.pipeline import build_problem
    w = CASES[request.param]
    prob = build_problem(w, geneo=False)
    s = pkg.Solver.from_workload(w, geneo=0, precision=pkg.PREC_FP32)
    yield request.param, w, prob, s
    s.close()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def test_split_local_solve(mcase):
    import paper_2311_18783_gb300 as pkg
    name, w, prob, s = mcase
    r = np.random.default_rng(31).standard_normal(s.n)
    out = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.local_solve(dev(r), out)
    ref = prob.M.local(r)
    err = np.abs(host(out) - ref).max() / np.abs(ref).max()
    # float32 storage of C_j plus the float64 inverse's own kappa * u error
    from test_gpu_parity import _kappa_local, U
    assert err <= 1e-5 + 1e3 * _kappa_local(prob) * U, err
    # the float64 factors are kept and selectable
    s.use_precision(pkg.PREC_FP64)
    s.local_solve(dev(r), out)
    assert np.abs(host(out) - ref).max() / np.abs(ref).max() <= 1e3 * _kappa_local(prob) * U
    s.use_precision(pkg.PREC_FP32)


def test_mixed_pcg(mcase):
    import paper_2311_18783_gb300 as pkg
    from oracle.solver import direct_solve
    name, w, prob, s = mcase
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(w.f_slot[0], b)
    x = torch.zeros_like(b)
    s.use_precision(pkg.PREC_FP64)
    i64 = s.solve(b, x, tol=1e-10, maxit=500)
    s.use_precision(pkg.PREC_FP32)
    x.zero_()
    i32 = s.solve(b, x, tol=1e-10, maxit=500)
    assert i32["status"] == 0 and i32["relres"] <= 1e-10
    assert abs(i32["iters"] - i64["iters"]) <= 2
    xs = direct_solve(prob.A, prob.b[0])
    ev = np.linalg.eigvalsh(prob.A.toarray())
    err = np.linalg.norm(host(x) - xs) / np.linalg.norm(xs)
    assert err <= max(2 * (ev[-1] / ev[0]) * 1e-10, 1e-12)


def test_gradient_part_in_float32(mcase):
    """S_j^-1 rounded to float32 as well (geneo_use_gradient_precision): the
    split local solve against the oracle's local solve within the float32
    storage error of C_j and S_j^-1 relative to the gradient part, the
    split inverse stays SPD (PCG converges), and PCG keeps the float64
    iteration count (+-2) and the solution bound of the float32 split."""
    import paper_2311_18783_gb300 as pkg
    from oracle.solver import direct_solve
    from test_gpu_parity import _kappa_local, U
    name, w, prob, s = mcase
    s.use_precision(pkg.PREC_FP32)
    s.use_gradient_precision(pkg.PREC_FP32)
    try:
        r = np.random.default_rng(31).standard_normal(s.n)
        out = torch.empty(s.n, dtype=torch.float64, device="cuda")
        s.local_solve(dev(r), out)
        ref = prob.M.local(r)
        err = np.abs(host(out) - ref).max() / np.abs(ref).max()
        assert err <= 1e-5 + 1e3 * _kappa_local(prob) * U, err
        b = torch.empty(s.n, dtype=torch.float64, device="cuda")
        s.assemble_rhs(w.f_slot[0], b)
        x = torch.zeros_like(b)
        i32 = s.solve(b, x, tol=1e-10, maxit=500)
        s.use_gradient_precision(pkg.PREC_FP64)
        x64 = torch.zeros_like(b)
        i64 = s.solve(b, x64, tol=1e-10, maxit=500)
        assert i32["status"] == 0 and abs(i32["iters"] - i64["iters"]) <= 2
        xs = direct_solve(prob.A, prob.b[0])
        ev = np.linalg.eigvalsh(prob.A.toarray())
        e = np.linalg.norm(host(x) - xs) / np.linalg.norm(xs)
        assert e <= max(2 * (ev[-1] / ev[0]) * 1e-10, 1e-12)
    finally:
        s.use_gradient_precision(pkg.PREC_FP64)
