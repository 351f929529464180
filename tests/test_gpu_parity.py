"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Integer set-up data (mesh, boundary, unknown numbering, CSR pattern,
subdomain index sets, partition of unity owners, split near-kernel columns,
k0, k1) must match bit for bit.  Floating-point results are compared element
by element with tolerances derived from the arithmetic:
* assembly and SpMV: sums of at most ~100 float64 terms -> 1e-14 relative;
* explicit inverses (tiled Cholesky) applied to a vector: forward error
  <= c * kappa(A_i) * u with u = 2^-53; the tests use c = 1e3;
* PCG solutions at relative residual 1e-12: ||x - x*|| / ||x*|| <=
  kappa(A) * 1e-12, and at most 1e-8 on the well-conditioned cases; with
  refinement on accurate residuals at most 1e-8 on every case.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _pkg():
    import paper_2311_18783_gb300 as pkg
    pkg.load_library()
    return pkg


def hetero_box(seed=0, gamma=1e-3, parts=(3, 2, 1), overlap=1, n=(10, 8, 6),
               holes=(((4, 6), (3, 5), (0, 6)),)):
    rng = np.random.default_rng(seed)
    nc = n[0] * n[1] * n[2]
    return W.box(*n, parts=parts, overlap=overlap, gamma=gamma,
                 mu_inv=10.0 ** rng.uniform(0, 2, nc), eps=10.0 ** rng.uniform(-0.5, 0.5, nc),
                 holes=holes, f='random', seed=seed, tau=0.1)


CASES = {
    "cube8": lambda: W.unit_cube_8(),
    "hetero_hole": lambda: hetero_box(),
    "overlap2": lambda: hetero_box(seed=1, parts=(2, 2, 1), overlap=2, n=(9, 9, 5), holes=()),
    "one_sub": lambda: hetero_box(seed=2, parts=(1, 1, 1), n=(5, 4, 4), holes=()),
    "ragged_beam": lambda: W.box(13, 3, 3, h=1 / 3, parts=(4, 1, 1), overlap=1, gamma=0.5,
                                  f=(0.2, -1.0, 0.7)),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    from oracle.pipeline import build_problem
    pkg = _pkg()
    w = CASES[request.param]()
    prob = build_problem(w, geneo=False)
    s = pkg.Solver.from_workload(w, geneo=0)
    yield request.param, w, prob, s
    s.close()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_integer_topology_bit_exact(case):
    name, w, prob, s = case
    m, dec = prob.mesh, prob.dec
    assert np.array_equal(s.export("edges").reshape(-1, 2), m.edges)
    assert np.array_equal(s.export("dir_edge").astype(bool), m.dir_edge)
    assert np.array_equal(s.export("dof_edge"), m.dof_edge)
    assert np.array_equal(s.export("dof_vert"), m.dof_vert)
    A = prob.A
    assert np.array_equal(s.export("A_rowptr"), A.indptr)
    assert np.array_equal(s.export("A_col"), A.indices)
    noff = s.export("N_off")
    nidx = s.export("N_idx")
    assert len(noff) == dec.nsub + 1
    for i in range(dec.nsub):
        assert np.array_equal(nidx[noff[i]:noff[i + 1]], dec.N[i])
    assert np.array_equal(s.export("owner"), dec.owner)
    assert np.array_equal(s.export("snk_sub"), np.array([c[0] for c in prob.snk], np.int32))
    assert np.array_equal(s.export("snk_vert"), np.array([c[1] for c in prob.snk], np.int32))
    from oracle.dd import k0, k1
    assert list(s.export("k0k1")) == [k0(A, dec), k1(dec)]


def test_assembly_and_rhs(case):
    name, w, prob, s = case
    A = prob.A
    assert rel(s.export("A_val"), A.data) <= 1e-14
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(w.f_slot[0], b)
    assert rel(host(b), prob.b[0]) <= 1e-13


def test_spmv(case):
    name, w, prob, s = case
    x = np.random.default_rng(7).standard_normal(s.n)
    y = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.spmv(dev(x), y)
    assert rel(host(y), prob.A @ x) <= 1e-14


def _kappa_local(prob):
    k = 1.0
    for Ni in prob.dec.N:
        ev = np.linalg.eigvalsh(prob.A[Ni][:, Ni].toarray())
        k = max(k, ev[-1] / ev[0])
    return k


def test_local_solve(case):
    """w = sum_i R_i^T A_i^-1 R_i r (Sec. 2, eq. "AS")."""
    name, w, prob, s = case
    r = np.random.default_rng(3).standard_normal(s.n)
    out = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.local_solve(dev(r), out)
    ref = prob.M.local(r)
    assert rel(host(out), ref) <= 1e3 * _kappa_local(prob) * U


def test_coarse_solve(case):
    """y = Z E^-1 Z^T r with the split near-kernel Z (same columns)."""
    name, w, prob, s = case
    r = np.random.default_rng(4).standard_normal(s.n)
    out = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.coarse_solve(dev(r), out)
    ref = prob.M.coarse(r)
    Z = prob.Z.toarray()
    ev = np.linalg.eigvalsh(Z.T @ (prob.A @ Z))
    assert rel(host(out), ref) <= 1e3 * (ev[-1] / ev[0]) * U


def test_apply_preconditioner(case):
    """z = M^-1_AS,2 r (Sec. 2, eq. "AS2").  s = r - A y0 is formed with the
    assembled A, where the coarse part y0 carries gradients that A nearly
    annihilates; the rounding of that product is amplified by
    rho = || |A| |y0| || / ||r|| on both sides, so the bound includes rho."""
    name, w, prob, s = case
    r = np.random.default_rng(5).standard_normal(s.n)
    out = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.apply_preconditioner(dev(r), out)
    ref = prob.M.apply(r)
    Z = prob.Z.toarray()
    ev = np.linalg.eigvalsh(Z.T @ (prob.A @ Z))
    k = max(_kappa_local(prob), ev[-1] / ev[0])
    y0 = prob.M.coarse(r)
    absA = abs(prob.A)
    rho = max(1.0, np.abs(absA @ np.abs(y0)).max() / np.abs(r).max())
    assert rel(host(out), ref) <= 1e4 * k * rho * U


def test_pcg_solution(case):
    """PCG to 1e-12 reaches the oracle's accurate solution (sparse LU plus
    refinement with extended residuals) within kappa(A) * 1e-12 and takes the
    oracle's iteration count (+-1); with two refinement steps (accurate
    residuals, geneo_solve_refined) the forward error is at most 1e-8 on
    every case, however large kappa(A) is."""
    from oracle.solver import refined_direct_solve, pcg
    name, w, prob, s = case
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(w.f_slot[0], b)
    x = torch.zeros_like(b)
    info = s.solve(b, x, tol=1e-12, maxit=500)
    assert info["status"] == 0 and info["relres"] <= 1e-12
    xs, _ = refined_direct_solve(prob.A, prob.b[0], steps=3)
    ev = np.linalg.eigvalsh(prob.A.toarray()) if s.n < 4000 else None
    kappa = ev[-1] / ev[0] if ev is not None else 1e6
    err = np.linalg.norm(host(x) - xs) / np.linalg.norm(xs)
    assert err <= max(2 * kappa * 1e-12, 1e-13)
    if kappa < 1e4:
        assert err <= 1e-8
    ro = pcg(prob.A, prob.b[0], prob.M.apply, tol=1e-12, maxit=500)
    assert abs(ro.iters - info["iters"]) <= 1
    xr = torch.zeros_like(b)
    ir = s.solve_refined(b, xr, tol=1e-12, maxit=500, nref=2)
    assert ir["status"] == 0
    err_r = np.linalg.norm(host(xr) - xs) / np.linalg.norm(xs)
    print(f"{name}: kappa {kappa:.2e}, PCG error {err:.2e}, refined {err_r:.2e}")
    assert err_r <= 1e-8


def test_pcg_balanced_form(case):
    """The balanced form (x0 = Z E^-1 Z^T b, one coarse solve per apply)
    against the oracle's balanced PCG: the same iteration count (+-1), and
    against the literal form: the same iteration count (+-1) and the same
    solution within kappa(A) * 1e-12."""
    from oracle.pipeline import solve as oracle_solve
    name, w, prob, s = case
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(w.f_slot[0], b)
    x0, x1 = torch.zeros_like(b), torch.zeros_like(b)
    i0 = s.solve(b, x0, tol=1e-12, maxit=500)
    s.use_balanced(True)
    try:
        i1 = s.solve(b, x1, tol=1e-12, maxit=500)
    finally:
        s.use_balanced(False)
    assert i1["status"] == 0 and abs(i1["iters"] - i0["iters"]) <= 1
    ob = oracle_solve(prob, tol=1e-12, maxit=500, balanced=True)
    assert abs(ob.iters - i1["iters"]) <= 1
    ev = np.linalg.eigvalsh(prob.A.toarray()) if s.n < 4000 else None
    kappa = ev[-1] / ev[0] if ev is not None else 1e6
    assert np.linalg.norm(host(x1) - host(x0)) <= max(4 * kappa * 1e-12, 1e-13) * \
        np.linalg.norm(host(x0))


def test_gmres_right_preconditioned(case):
    """Right-preconditioned GMRES with M^-1_AS,2 (Sec. 4's Krylov method)
    against the oracle's GMRES: the same Arnoldi step count (+-1) to a true
    relative residual of 1e-8 (GMRES stops on ||b - A x||, whose float64
    value cannot fall below about u ||A|| ||x|| / ||b||, 1e-10 on the small
    gamma cases), and the solution within 2 kappa(A) 1e-8 of the oracle's
    accurate one."""
    from oracle.solver import gmres_right, refined_direct_solve
    name, w, prob, s = case
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(w.f_slot[0], b)
    x = torch.zeros_like(b)
    info = s.solve_gmres(b, x, tol=1e-8, maxit=500, restart=60)
    assert info["status"] == 0 and info["relres"] <= 1e-8
    ro = gmres_right(prob.A, prob.b[0], prob.M.apply, tol=1e-8, maxit=500, restart=60)
    assert ro.relres <= 1e-8 and abs(ro.iters - info["iters"]) <= 1
    xs, _ = refined_direct_solve(prob.A, prob.b[0], steps=3)
    ev = np.linalg.eigvalsh(prob.A.toarray()) if s.n < 4000 else None
    kappa = ev[-1] / ev[0] if ev is not None else 1e6
    err = np.linalg.norm(host(x) - xs) / np.linalg.norm(xs)
    assert err <= max(2 * kappa * 1e-8, 1e-13)


def test_solve_host_matches_device(case):
    name, w, prob, s = case
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(w.f_slot[0], b)
    x = torch.zeros_like(b)
    info = s.solve(b, x, tol=1e-10, maxit=500)
    xh, info2 = s.solve_host(host(b), tol=1e-10, maxit=500)
    assert info2["iters"] == info["iters"]
    assert np.array_equal(xh.numpy(), host(x))


def test_invalid_arguments_rejected():
    pkg = _pkg()
    w = W.box(4, 4, 4, parts=(2, 2, 2))
    with pytest.raises(pkg.GeneoError) as e:
        pkg.Solver(4, 4, 4, 0.25, w.active, w.mu_inv, w.eps, -1.0, (2, 2, 2), 1, 0.1, geneo=0)
    assert e.value.status == -1
    with pytest.raises(pkg.GeneoError):
        pkg.Solver(4, 4, 4, 0.25, w.active, w.mu_inv, w.eps, 1.0, (2, 2, 2), 0, 0.1, geneo=0)
