"""Independent problems in one context (workloads.compose stacks them along z
with an inactive cell layer between them; each keeps its own boxes through an
explicit cell partition).  A, Z and M^-1_AS,2 are then block diagonal over
the problems (Sec. 2-3: every subdomain and every coarse column lies in one
problem), so the segmented PCG must give, per problem:
* the problem's own right-hand side (1e-14 relative, same float64 sums),
* its direct solution within 2 kappa tol (kappa from the oracle's spectrum),
* the iteration count of a separate solve of that problem (+-1; the dot
  products are summed in another order),
and a problem with b = 0 stops at once with x = 0."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H = 1.0 / 6


def _problems():
    rng = np.random.default_rng(5)
    p0 = W.box(6, 6, 6, h=H, parts=(2, 1, 1), overlap=1, gamma=1e-2,
               mu_inv=10.0 ** rng.uniform(0, 2, 216), f='random', seed=1)
    p1 = W.box(5, 4, 4, h=H, parts=(1, 2, 1), overlap=1, gamma=1.0, f='random', seed=2)
    p2 = W.box(4, 4, 3, h=H, parts=(2, 1, 1), overlap=1, gamma=0.5, f=(0.0, 0.0, 0.0))
    p3 = W.box(6, 5, 5, h=H, parts=(1, 1, 2), overlap=1, gamma=1e-3,
               eps=10.0 ** rng.uniform(-1, 1, 150), f='random', seed=3)
    return [p0, p1, p2, p3]


@pytest.fixture(scope="module")
def batch():
    import paper_2311_18783_gb300 as pkg
    ps = _problems()
    c = W.compose(ps)
    s = pkg.Solver.from_workload(c)
    yield pkg, ps, c, s
    s.close()


def _dofs_of(s):
    e = s.export("edges").reshape(-1, 2)
    return e[s.export("dof_edge")]


def _local_map(c, w, zoff, pairs):
    """composite vertex pairs -> the problem's own vertex pairs."""
    def conv(v):
        i = v % (c.nx + 1)
        j = (v // (c.nx + 1)) % (c.ny + 1)
        k = v // ((c.nx + 1) * (c.ny + 1)) - zoff
        assert np.all((i <= w.nx) & (j <= w.ny) & (k >= 0) & (k <= w.nz))
        return i + (w.nx + 1) * (j + (w.ny + 1) * k)
    return np.stack([conv(pairs[:, 0]), conv(pairs[:, 1])], axis=1)


def test_segments_match_separate_problems(batch):
    from oracle.pipeline import build_problem
    from oracle.solver import direct_solve
    pkg, ps, c, s = batch
    off = s.export("seg_off")
    assert len(off) == len(ps) + 1
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(c.f_slot[0], b)
    x = torch.full_like(b, 7.0)
    tol = 1e-10
    st, infos = s.solve_segments(b, x, tol=tol, maxit=500)
    assert st == 0
    bh, xh = b.cpu().numpy(), x.cpu().numpy()
    pairs = _dofs_of(s)
    for p, (w, zo) in enumerate(zip(ps, c.meta["zoff"])):
        prob = build_problem(w, geneo=False)
        lo, hi = off[p], off[p + 1]
        assert hi - lo == prob.A.shape[0]
        loc = _local_map(c, w, zo, pairs[lo:hi])
        own = prob.mesh.edges[prob.mesh.dof_edge]
        row = {(int(a), int(bb)): r for r, (a, bb) in enumerate(own.tolist())}
        perm = np.array([row[(int(a), int(bb))] for a, bb in loc.tolist()])
        assert np.array_equal(np.sort(perm), np.arange(hi - lo))
        bp = prob.b[0][perm]
        assert np.abs(bh[lo:hi] - bp).max() <= 1e-14 * max(np.abs(bp).max(), 1e-300)
        if not np.any(bp):
            assert infos[p]["iters"] == 0 and infos[p]["relres"] == 0.0
            assert not np.any(xh[lo:hi])
            continue
        assert infos[p]["relres"] <= tol
        xs = direct_solve(prob.A, prob.b[0])[perm]
        ev = np.linalg.eigvalsh(prob.A.toarray())
        err = np.linalg.norm(xh[lo:hi] - xs) / np.linalg.norm(xs)
        assert err <= max(2 * ev[-1] / ev[0] * tol, 1e-13)
        # the same problem alone
        sp = pkg.Solver.from_workload(w)
        bq = torch.empty(sp.n, dtype=torch.float64, device="cuda")
        sp.assemble_rhs(w.f_slot[0], bq)
        xq = torch.zeros_like(bq)
        info = sp.solve(bq, xq, tol=tol, maxit=500)
        sp.close()
        print(f"problem {p}: n={hi - lo} segmented {infos[p]['iters']} alone {info['iters']}")
        assert abs(info["iters"] - infos[p]["iters"]) <= 1


def test_segments_graph_equals_plain_launches(batch):
    """The segmented PCG iteration replayed as a CUDA graph gives the same
    iterates, bit for bit, as plain launches (a context with use_graph = 0),
    in the literal and the balanced form."""
    import paper_2311_18783_gb300 as pkg
    pkg_, ps, c, s = batch
    s0 = pkg.Solver.from_workload(c, use_graph=0)
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(c.f_slot[0], b)
    for bal in (False, True):
        s.use_balanced(bal)
        s0.use_balanced(bal)
        x1, x0 = torch.zeros_like(b), torch.zeros_like(b)
        st1, i1 = s.solve_segments(b, x1, tol=1e-10, maxit=500)
        st0, i0 = s0.solve_segments(b, x0, tol=1e-10, maxit=500)
        assert st1 == st0 == 0
        assert [q["iters"] for q in i1] == [q["iters"] for q in i0]
        assert torch.equal(x1, x0)
    s.use_balanced(False)
    s0.close()


def test_segments_rejected_when_not_contiguous():
    """Two components side by side along x interleave in the unknown
    numbering: the segmented solve refuses with STATE."""
    import paper_2311_18783_gb300 as pkg
    w = W.box(5, 3, 3, h=H, parts=(2, 1, 1), overlap=1, holes=(((2, 3), (0, 3), (0, 3)),),
              f='random', seed=4)
    s = pkg.Solver.from_workload(w)
    b = torch.ones(s.n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(pkg.GeneoError) as e:
        s.solve_segments(b, x)
    assert e.value.status == -7  # GENEO_ERR_STATE
    s.close()


def test_many_problems_subset():
    """The batching workload's own problems (n^3 unit cubes with holes, mu^-1
    in {1, 1e2, 1e4} on blocks, gamma log-uniform in [1e-6, 1], 8-64 boxes
    each), four of those with n <= 10, mapped onto one cell size.  Two of
    them hold a box whose edges all join boundary vertices (no gradient
    column in S_j); every component converges.  Iteration counts equal the
    separate solve (+-1) for gamma >= 1e-3 (measured 55/55); below that the
    local eigensolves stop at their iteration limit with seed-dependent
    results (the composite numbers its subdomains differently), so the
    counts are printed, not compared (measured 197/196 and 165/157)."""
    import paper_2311_18783_gb300 as pkg
    ps = [w for w in W.many_problems(256, seed=3) if w.nx <= 10][2:6]
    for w in ps:
        w.f_slot = W.box(w.nx, w.ny, w.nz, h=w.hx, f='random', seed=w.nx).f_slot
    c = W.compose(ps)
    s = pkg.Solver.from_workload(c)
    off = s.export("seg_off")
    assert len(off) == len(ps) + 1
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(c.f_slot[0], b)
    x = torch.zeros_like(b)
    st, infos = s.solve_segments(b, x, tol=1e-8, maxit=500)
    assert st == 0
    for p, w in enumerate(ps):
        sp = pkg.Solver.from_workload(w)
        assert sp.n == off[p + 1] - off[p]
        bq = torch.empty(sp.n, dtype=torch.float64, device="cuda")
        sp.assemble_rhs(w.f_slot[0], bq)
        assert torch.allclose(bq, b[off[p]:off[p + 1]], rtol=1e-12, atol=1e-14 * bq.abs().max())
        xq = torch.zeros_like(bq)
        info = sp.solve(bq, xq, tol=1e-8, maxit=500)
        sp.close()
        print(f"{w.name} parts {w.parts} gamma {w.gamma:.1e}: segmented {infos[p]['iters']} "
              f"alone {info['iters']}")
        assert infos[p]["relres"] <= 1e-8
        if w.gamma >= 1e-3:
            assert abs(info["iters"] - infos[p]["iters"]) <= 1
    s.close()

