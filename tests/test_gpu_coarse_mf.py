"""Sparse coarse solve: multifrontal Cholesky of E = Z^T A Z on a nested
dissection of the near-kernel vertices (Sec. 2, eq. "AS2" needs E^-1 only as
a solve).  Compared with the oracle's coarse solve y = Z E^-1 Z^T r and with
the library's explicit dense E^-1 on coarse spaces of a few thousand columns,
so that the elimination tree has several levels, fronts with update rows and
extend-adds over several children.  Tolerance: forward error of a Cholesky
solve, 1e3 * kappa(E) * u.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _pkg():
    import paper_2311_18783_gb300 as pkg
    pkg.load_library()
    return pkg


def _hetero(n, parts, seed, holes=(), gamma=1e-2):
    rng = np.random.default_rng(seed)
    nc = n[0] * n[1] * n[2]
    return W.box(*n, parts=parts, overlap=1, gamma=gamma,
                 mu_inv=10.0 ** rng.uniform(0, 2, nc), eps=10.0 ** rng.uniform(-0.5, 0.5, nc),
                 holes=holes, f='random', seed=seed)


# (workload, leaf size of the nested dissection); small leaves give deep
# trees with many fronts on problems the oracle factors in seconds
CASES = {
    # about 1000 columns, separators in all three directions, a hole
    "box14": (lambda: _hetero((14, 10, 8), (3, 3, 2), 11, holes=(((5, 9), (3, 7), (0, 8)),)), 24),
    # default leaf size: two levels
    "box14_leaf256": (lambda: _hetero((14, 10, 8), (3, 3, 2), 11,
                                      holes=(((5, 9), (3, 7), (0, 8)),)), 0),
    # long thin beam: a chain of small separators along x
    "beam40": (lambda: _hetero((40, 4, 3), (8, 1, 1), 12), 16),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    from oracle.pipeline import build_problem
    pkg = _pkg()
    make, leaf = CASES[request.param]
    w = make()
    prob = build_problem(w, geneo=False)
    s_mf = pkg.Solver.from_workload(w, geneo=0, coarse_leaf=leaf)
    s_dn = pkg.Solver.from_workload(w, geneo=0, coarse_dense=1)
    yield request.param, w, prob, s_mf, s_dn
    s_mf.close()
    s_dn.close()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _kappa_E(prob):
    Z = prob.Z.toarray()
    ev = np.linalg.eigvalsh(Z.T @ (prob.A @ Z))
    return ev[-1] / ev[0]


def test_sizes(case):
    name, w, prob, s_mf, s_dn = case
    q_mf, q_dn = s_mf.query(), s_dn.query()
    assert q_mf["n0"] == q_dn["n0"] == prob.Z.shape[1]
    assert q_mf["n0"] > 200
    # tiny trees pad every front to 64-wide tiles, so the sparse factor is
    # only smaller than the dense inverse on large coarse spaces
    assert q_mf["coarse_factor_bytes"] > 0 and q_dn["coarse_factor_bytes"] > 0


def test_coarse_solve_vs_oracle_and_dense(case):
    name, w, prob, s_mf, s_dn = case
    k = _kappa_E(prob)
    for seed in (0, 1):
        r = np.random.default_rng(seed).standard_normal(s_mf.n)
        y_mf = torch.empty(s_mf.n, dtype=torch.float64, device="cuda")
        y_dn = torch.empty_like(y_mf)
        s_mf.coarse_solve(dev(r), y_mf)
        s_dn.coarse_solve(dev(r), y_dn)
        ref = prob.M.coarse(r)
        assert rel(host(y_mf), ref) <= 1e3 * k * U
        assert rel(host(y_mf), host(y_dn)) <= 1e3 * k * U


def test_coarse_backward_error(case):
    """Backward stability of the sparse Cholesky solve, independent of
    kappa(E): with u = (Z^T Z)^-1 Z^T y recovered from y = Z u,
    ||E u - Z^T r|| <= 10 n0 u ||E|| ||u|| (E by the curl route, as the
    oracle forms it).  A dropped extend-add or a wrong update row gives an
    O(1) residual."""
    import scipy.sparse.linalg as spla
    from oracle.coarse import coarse_matrix
    name, w, prob, s_mf, s_dn = case
    Z = prob.Z.tocsc()
    E = coarse_matrix(prob.mesh, w, Z)
    E = E.toarray() if hasattr(E, "toarray") else np.asarray(E)
    n0 = E.shape[0]
    normE = np.linalg.norm(E, 2)
    r = np.random.default_rng(3).standard_normal(s_mf.n)
    y = torch.empty(s_mf.n, dtype=torch.float64, device="cuda")
    s_mf.coarse_solve(dev(r), y)
    u = spla.spsolve((Z.T @ Z).tocsc(), Z.T @ host(y))
    res = np.linalg.norm(E @ u - Z.T @ r)
    assert res <= 10 * n0 * U * normE * np.linalg.norm(u)


def test_coarse_solve_repeatable(case):
    """Split-K partials are summed in slot order, not by atomics on the
    values: two calls give identical bits."""
    name, w, prob, s_mf, s_dn = case
    r = dev(np.random.default_rng(7).standard_normal(s_mf.n))
    a = torch.empty_like(r)
    b = torch.empty_like(r)
    s_mf.coarse_solve(r, a)
    s_mf.coarse_solve(r, b)
    assert torch.equal(a, b)


def test_pcg_iterations_match_dense(case):
    name, w, prob, s_mf, s_dn = case
    b = torch.empty(s_mf.n, dtype=torch.float64, device="cuda")
    s_mf.assemble_rhs(w.f_slot[0], b)
    x1 = torch.zeros_like(b)
    x2 = torch.zeros_like(b)
    i1 = s_mf.solve(b, x1, tol=1e-10, maxit=500)
    i2 = s_dn.solve(b, x2, tol=1e-10, maxit=500)
    assert i1["status"] == 0 and i2["status"] == 0
    assert abs(i1["iters"] - i2["iters"]) <= 1
    assert rel(host(x1), host(x2)) <= 1e-7


def test_single_launch_equals_level_launches(case):
    """The coarse solve as one cooperative launch (grid barriers between the
    level-by-level steps, factor tiles staged by bulk copies) computes every
    tile task in the same order as one launch per level and phase: identical
    bits, for one column and inside a block preconditioner apply of three
    columns."""
    name, w, prob, s_mf, s_dn = case
    r = dev(np.random.default_rng(11).standard_normal(s_mf.n))
    a = torch.empty_like(r)
    b = torch.empty_like(r)
    try:
        s_mf.use_persistent_coarse(True)
        s_mf.coarse_solve(r, a)
        s_mf.use_persistent_coarse(False)
        s_mf.coarse_solve(r, b)
        assert torch.equal(a, b)
        R = dev(np.random.default_rng(12).standard_normal((3, s_mf.n)))
        Z1 = torch.empty_like(R)
        Z2 = torch.empty_like(R)
        s_mf.use_persistent_coarse(True)
        s_mf.apply_preconditioner_block(R, Z1)
        s_mf.use_persistent_coarse(False)
        s_mf.apply_preconditioner_block(R, Z2)
        assert torch.equal(Z1, Z2)
    finally:
        s_mf.use_persistent_coarse(True)


def test_single_launch_pcg_graph(case):
    """PCG replays its iteration as a CUDA graph whose key includes the
    coarse kernel shape: switching between the two shapes gives the same
    iterates bit for bit, in both PCG forms."""
    name, w, prob, s_mf, s_dn = case
    bvec = torch.empty(s_mf.n, dtype=torch.float64, device="cuda")
    s_mf.assemble_rhs(w.f_slot[0], bvec)
    try:
        for balanced in (False, True):
            s_mf.use_balanced(balanced)
            xs, its = [], []
            for persistent in (True, False, True):
                s_mf.use_persistent_coarse(persistent)
                x = torch.zeros_like(bvec)
                info = s_mf.solve(bvec, x, tol=1e-10, maxit=500)
                assert info["status"] == 0
                xs.append(x)
                its.append(info["iters"])
            assert its[0] == its[1] == its[2]
            assert torch.equal(xs[0], xs[1]) and torch.equal(xs[0], xs[2])
    finally:
        s_mf.use_persistent_coarse(True)
        s_mf.use_balanced(False)
