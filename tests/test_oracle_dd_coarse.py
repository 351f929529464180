"""Pins of the oracle's decomposition, coarse space, preconditioner and PCG
against the paper's identities and condition-number statements (no GPU)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import workloads as W
from oracle.mesh import build_mesh, gradient_dofs
from oracle.fem import assemble_A, local_element_A, assemble_rhs
from oracle.dd import decompose, k0, k1, restriction, local_dirichlet, local_neumann
from oracle.coarse import (snk_columns, assemble_Z, local_gradient, xi_projector,
                           local_gevp, geneo_columns)
from oracle.solver import build_preconditioner, pcg, direct_solve
from oracle.pipeline import build_problem, solve


def small(n=(6, 5, 4), parts=(2, 2, 1), overlap=1, gamma=1e-2, holes=(), seed=0, mu=None,
          tau=0.1):
    rng = np.random.default_rng(seed)
    nc = n[0] * n[1] * n[2]
    mu_inv = mu if mu is not None else 10.0 ** rng.uniform(0, 2, nc)
    return W.box(*n, parts=parts, overlap=overlap, gamma=gamma, mu_inv=mu_inv,
                 eps=10.0 ** rng.uniform(-0.5, 0.5, nc), holes=holes, f='random',
                 seed=seed, tau=tau)


def setup(w, pou="boolean"):
    m = build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active)
    A = assemble_A(m, w)
    AT = local_element_A(m, w)
    dec = decompose(m, w.parts, w.overlap, pou=pou)
    return m, A, AT, dec


@pytest.mark.parametrize("pou", ["boolean", "core"])
def test_partition_of_unity(pou):
    """sum_i R_i^T D_i R_i = I (Sec. 2, eq. "PoU"), D_i >= 0."""
    w = small(holes=[((2, 4), (2, 3), (0, 4))])
    m, A, AT, dec = setup(w, pou)
    n = A.shape[0]
    S = sum(restriction(dec, i, n).T @ sp.diags(dec.D[i]) @ restriction(dec, i, n)
            for i in range(dec.nsub))
    assert all((d >= 0).all() for d in dec.D)
    assert np.abs(S.toarray() - np.eye(n)).max() <= 4 * np.finfo(float).eps


def test_neumann_sum_and_lemma_k1():
    """sum_i R_i^T A_i^Neu R_i = sum_T m_T A_T, which gives Lemma "Lemma_k1":
    sum_i (R_i U)^T A_i^Neu (R_i U) <= k1 U^T A U."""
    w = small(n=(6, 6, 3), parts=(3, 2, 1), overlap=1)
    m, A, AT, dec = setup(w)
    n = A.shape[0]
    S = sum(restriction(dec, i, n).T @ sp.csr_matrix(local_neumann(m, AT, dec, i)) @
            restriction(dec, i, n) for i in range(dec.nsub))
    # multiplicity-weighted assembly
    ntet = len(m.tets)
    mult = dec.cell_mult[m.tet_cell]
    from oracle.fem import assemble_edges, mirror_upper
    Aw = mirror_upper(assemble_edges(m, AT * mult[:, None, None])[m.dof_edge][:, m.dof_edge])
    assert np.abs((S - Aw).toarray()).max() <= 1e-12 * np.abs(Aw).max()
    kk1 = k1(dec)
    rng = np.random.default_rng(1)
    for _ in range(5):
        U = rng.standard_normal(n)
        lhs = sum(U[dec.N[i]] @ local_neumann(m, AT, dec, i) @ U[dec.N[i]] for i in range(dec.nsub))
        assert lhs <= kk1 * (U @ (A @ U)) * (1 + 1e-12)
    # A_i^Neu is SPD (gamma > 0) and A_i^Neu <= A_i in energy
    for i in range(dec.nsub):
        An = local_neumann(m, AT, dec, i)
        assert np.linalg.eigvalsh(An)[0] > 0
        Ai = local_dirichlet(A, dec, i)
        assert np.linalg.eigvalsh(Ai - An)[0] >= -1e-10 * np.abs(Ai).max()


def test_lemma_k0():
    """Lemma "Lemma_k0" with Q_i = R_i^T: |sum_i R_i^T U_i|_A^2 <= k0 sum_i |U_i|_{A_i}^2."""
    w = small(n=(6, 4, 4), parts=(3, 2, 1), overlap=1)
    m, A, AT, dec = setup(w)
    kk0 = k0(A, dec)
    assert 1 <= kk0 <= dec.nsub
    n = A.shape[0]
    rng = np.random.default_rng(2)
    for _ in range(5):
        Us = [rng.standard_normal(len(Ni)) for Ni in dec.N]
        v = np.zeros(n)
        for Ni, U in zip(dec.N, Us):
            v[Ni] += U
        rhs = sum(U @ local_dirichlet(A, dec, i) @ U for i, U in enumerate(Us))
        assert v @ (A @ v) <= kk0 * rhs * (1 + 1e-12)


def test_snk_full_rank_boolean_and_contains_local_gradients():
    """Z_G has full rank (Sec. 3.2 requires a full-rank Z) and spans
    R_i^T D_i G_i for every i (Sec. 2, definition "near-kernelCS")."""
    w = small(n=(6, 6, 4), parts=(2, 2, 2), overlap=1, holes=[((2, 4), (2, 4), (0, 4))])
    m, A, AT, dec = setup(w)
    Z = assemble_Z(A.shape[0], snk_columns(m, dec)).toarray()
    s = np.linalg.svd(Z, compute_uv=False)
    assert s[-1] > 1e-3 * s[0]
    G = gradient_dofs(m).toarray()
    for i in range(dec.nsub):
        Ni = dec.N[i]
        V = np.zeros((A.shape[0], G.shape[1]))
        V[Ni] = dec.D[i][:, None] * G[Ni]
        coef, *_ = np.linalg.lstsq(Z, V, rcond=None)
        assert np.abs(Z @ coef - V).max() < 1e-10
    # the global gradient is inside V_G (G in V_G, Sec. 2)
    coef, *_ = np.linalg.lstsq(Z, G, rcond=None)
    assert np.abs(Z @ coef - G).max() < 1e-10


def test_core_pou_snk_is_rank_deficient():
    """With the core-edge partition of unity the per-(i, v) columns are
    linearly dependent across subdomains even after removing floating and
    duplicate columns; this is why the Boolean partition of unity is used."""
    w = W.unit_cube_8()
    m, A, AT, dec = setup(w, "core")
    Z = assemble_Z(A.shape[0], snk_columns(m, dec)).toarray()
    s = np.linalg.svd(Z, compute_uv=False)
    assert s[-1] < 1e-12 * s[0]


def test_xi_projector_properties():
    """xi_0i is the A_i-orthogonal projection on range(G_i) and
    B^dagger = (I - xi) A_i^-1 inverts A_i on its A_i-orthogonal complement
    (Sec. 2, eq. "inverseBw")."""
    w = small(n=(6, 5, 4), parts=(2, 2, 1), overlap=1)
    m, A, AT, dec = setup(w)
    for i in range(dec.nsub):
        Ai = local_dirichlet(A, dec, i)
        Gi, kept = local_gradient(m, dec, i)
        assert np.linalg.matrix_rank(Gi) == Gi.shape[1]
        xi = xi_projector(Ai, Gi)
        sc = np.abs(xi).max()
        assert np.abs(xi @ xi - xi).max() < 1e-10 * sc
        assert np.abs(Ai @ xi - xi.T @ Ai).max() < 1e-10 * np.abs(Ai).max() * sc
        assert np.abs((np.eye(len(Ai)) - xi) @ Gi).max() < 1e-10
        Bd = (np.eye(len(Ai)) - xi) @ np.linalg.inv(Ai)
        rng = np.random.default_rng(i)
        y = rng.standard_normal(len(Ai))
        # y in the complement: b_i(y, G_i c) = 0  <=>  G_i^T A_i y = 0 ... here
        # take y = A_i (I - xi) u, the image of the complement under A_i
        y = Ai @ ((np.eye(len(Ai)) - xi) @ y)
        u = Bd @ y
        assert np.abs(Gi.T @ Ai @ u).max() < 1e-8 * np.abs(u).max() * np.abs(Ai).max()
        assert np.abs(Ai @ u - y).max() < 1e-8 * np.abs(y).max()


def test_split_inverse_identities():
    """Identities the library's split local solves rest on (Sec. 2, eq.
    "inverseBw", with xi_i = G S^-1 G^T A_i a projection):
    * C = (I - xi) A_i^-1 = A_i^-1 - G S^-1 G^T, and C = (I - xi) C (I - xi)^T
      (the two-sided form applied to bfloat16 factors);
    * for any rho > 0, A~ = A_i (I + rho xi) = A_i + rho A_i G S^-1 G^T A_i is
      symmetric and A~^-1 = A_i^-1 - rho/(1+rho) G S^-1 G^T, so that
      C = A~^-1 - G S^-1 G^T / (1 + rho) (the gradient shift)."""
    w = small(n=(6, 5, 4), parts=(2, 2, 1), overlap=1)
    m, A, AT, dec = setup(w)
    for i in range(dec.nsub):
        Ai = local_dirichlet(A, dec, i)
        Gi, _ = local_gradient(m, dec, i)
        n = len(Ai)
        S = Gi.T @ Ai @ Gi
        GSG = Gi @ np.linalg.solve(S, Gi.T)
        xi = GSG @ Ai
        Ainv = np.linalg.inv(Ai)
        P = np.eye(n) - xi
        C = P @ Ainv
        sc = np.abs(Ainv).max()
        assert np.abs(C - (Ainv - GSG)).max() < 1e-9 * sc
        assert np.abs(C - P @ C @ P.T).max() < 1e-9 * sc
        assert np.abs(C @ Ai @ Gi).max() < 1e-9 * sc * np.abs(Ai).max()
        for rho in (0.5, 1e3):
            At = Ai + rho * Ai @ GSG @ Ai
            # rounding of the triple product: relative u kappa(S) rho
            assert np.abs(At - At.T).max() < 1e-8 * np.abs(At).max()
            assert np.abs(At - Ai @ (np.eye(n) + rho * xi)).max() < 1e-8 * np.abs(At).max()
            Atinv = np.linalg.inv(At)
            assert np.abs(Atinv - (Ainv - rho / (1 + rho) * GSG)).max() < 1e-6 * sc
            assert np.abs(C - (Atinv - GSG / (1 + rho))).max() < 1e-6 * sc


def test_gevp_count_by_inertia():
    """#{lambda > tau} of eq. "eigAtildeBAS" equals the number of positive
    eigenvalues of L - tau B (Sylvester), computed by an LDL^T inertia count
    independent of the eigensolver."""
    w = small(n=(6, 6, 4), parts=(2, 2, 1), overlap=1, gamma=1e-3)
    m, A, AT, dec = setup(w)
    for tau in (0.5, 2.0):
        for j in range(dec.nsub):
            g = local_gevp(m, w, A, AT, dec, j)
            Lm = g.L - tau * g.Aneu
            lu, d, perm = sla.ldl(0.5 * (Lm + Lm.T))
            evd = np.concatenate([np.linalg.eigvalsh(d[k:k + 2, k:k + 2]) if (
                k + 1 < len(d) and d[k + 1, k] != 0) else [d[k, k]] for k in _blocks(d)])
            assert int((evd > 0).sum()) == int((g.lam > tau).sum())
            # eigen-residual and B-orthonormality of the oracle's eigensolve
            V, lam = g.V[:, :5], g.lam[:5]
            R = g.L @ V - g.Aneu @ V * lam
            assert np.abs(R).max() < 1e-8 * np.abs(g.L).max()
            assert np.allclose(V.T @ g.Aneu @ V, np.eye(5), atol=1e-10)


def _blocks(d):
    k, out = 0, []
    while k < len(d):
        out.append(k)
        k += 2 if (k + 1 < len(d) and d[k + 1, k] != 0) else 1
    return out


def _dense_precond(prob):
    n = prob.A.shape[0]
    return np.column_stack([prob.M.apply(e) for e in np.eye(n)])


def test_preconditioner_identities():
    """M^-1 symmetric (eq. "AS2"); (I - P0) Z = 0; (I - P0) sum_i R_i^T D_i
    xi_0i R_i U = 0 (Sec. 3.1, proof of the stable decomposition)."""
    w = small(n=(6, 5, 4), parts=(2, 2, 1), overlap=1, tau=3.0)
    prob = build_problem(w, tau_convention="paper")
    assert len(prob.geneo) > 0
    A = prob.A.toarray()
    Minv = _dense_precond(prob)
    assert np.abs(Minv - Minv.T).max() < 1e-10 * np.abs(Minv).max()
    Z = prob.Z.toarray()
    E = Z.T @ A @ Z
    P0 = Z @ np.linalg.solve(E, Z.T @ A)
    assert np.abs((np.eye(len(A)) - P0) @ Z).max() < 1e-9
    rng = np.random.default_rng(3)
    U = rng.standard_normal(len(A))
    v = np.zeros(len(A))
    for i in range(prob.dec.nsub):
        Ai = local_dirichlet(prob.A, prob.dec, i)
        Gi, _ = local_gradient(prob.mesh, prob.dec, i)
        v[prob.dec.N[i]] += prob.dec.D[i] * (xi_projector(Ai, Gi) @ U[prob.dec.N[i]])
    assert np.abs((np.eye(len(A)) - P0) @ v).max() < 1e-9 * np.abs(v).max()


def test_exact_cases():
    """Z = I gives M^-1 = A^-1; one subdomain covering Omega gives A^-1."""
    w = small(n=(4, 4, 3), parts=(2, 1, 1), overlap=1)
    m, A, AT, dec = setup(w)
    n = A.shape[0]
    M = build_preconditioner(A, dec, sp.identity(n, format='csc'))
    r = np.random.default_rng(0).standard_normal(n)
    x = direct_solve(A, r)
    assert np.abs(M.apply(r) - x).max() < 1e-10 * np.abs(x).max()
    w1 = small(n=(4, 4, 3), parts=(1, 1, 1), overlap=1)
    p1 = build_problem(w1)
    assert np.abs(p1.M.apply(r) - x).max() < 1e-10 * np.abs(x).max()


@pytest.mark.parametrize("tau_p", [2.0, 3.0])
def test_condition_number_bound_geneo(tau_p):
    """Theorem (Sec. 3.2): the eigenvalues of M^-1_AS,2 A lie in
    [1/(1 + k1 tau), k0] (Lemma "surj_cont" gives the upper bound)."""
    w = small(n=(6, 4, 4), parts=(2, 2, 1), overlap=1, gamma=1e-3, tau=tau_p, seed=5)
    prob = build_problem(w, tau_convention="paper")
    A = prob.A.toarray()
    ev = np.sort(np.real(np.linalg.eigvals(_dense_precond(prob) @ A)))
    kk0, kk1 = k0(prob.A, prob.dec), k1(prob.dec)
    assert ev[-1] <= kk0 * (1 + 1e-8)
    assert ev[0] >= 1.0 / (1.0 + kk1 * tau_p) * (1 - 1e-8)


def test_condition_number_bound_snk_only():
    """Theorem (Sec. 3.1): with the SNK space alone the eigenvalues lie in
    [1/(1 + k1 tau0), k0] with tau0 of eq. "tauOneLevelAS"."""
    w = small(n=(6, 4, 4), parts=(2, 2, 1), overlap=1, gamma=1e-3, seed=6)
    prob = build_problem(w, geneo=False)
    m, A, AT, dec = prob.mesh, prob.A, prob.AT, prob.dec
    tau0 = max(local_gevp(m, w, A, AT, dec, j).lam[0] for j in range(dec.nsub))
    ev = np.sort(np.real(np.linalg.eigvals(_dense_precond(prob) @ A.toarray())))
    assert ev[-1] <= k0(A, dec) * (1 + 1e-8)
    assert ev[0] >= 1.0 / (1.0 + k1(dec) * tau0) * (1 - 1e-8)


def test_pcg_matches_direct_solve():
    w = small(n=(6, 6, 4), parts=(2, 2, 2), overlap=1, gamma=1e-4,
              holes=[((2, 4), (2, 4), (0, 4))])
    prob = build_problem(w)
    x = direct_solve(prob.A, prob.b[0])
    r = solve(prob, tol=1e-12, maxit=500)
    assert r.relres <= 1e-12
    ev = np.linalg.eigvalsh(prob.A.toarray())
    kappa = ev[-1] / ev[0]
    # forward error <= kappa(A) * relative residual
    assert np.linalg.norm(r.x - x) / np.linalg.norm(x) <= 2 * kappa * r.relres + 1e-12
    # the one-level method needs more iterations than the two-level one
    r1 = pcg(prob.A, prob.b[0], build_problem(w, coarse="none", geneo=False).M.apply, 1e-8)
    r2 = solve(prob, tol=1e-8)
    assert r2.iters <= r1.iters


def test_galerkin_through_curl_operator():
    """K = C^T C, and E = Z^T A Z computed element by element through C
    equals the assembled product; for pure gradients the curl-route K-part
    vanishes to rounding squared, far below the assembled residue."""
    from oracle.fem import curl_operator, assemble_K
    from oracle.coarse import galerkin
    w = small(n=(6, 5, 4), parts=(2, 2, 1), overlap=1, gamma=1e-2)
    m, A, AT, dec = setup(w)
    C = curl_operator(m, w)
    K = assemble_K(m, w)
    assert abs(C.T @ C - K).max() <= 1e-13 * abs(K).max()
    Z = assemble_Z(A.shape[0], snk_columns(m, dec))
    E1 = galerkin(m, w, Z)
    E2 = (Z.T @ (A @ Z)).toarray()
    assert np.abs(E1 - E2).max() <= 1e-12 * np.abs(A).max()
    G = gradient_dofs(m)
    CG = C @ G
    assert abs(CG.T @ CG).max() <= 1e-24 * abs(K).max()


def test_cell_partition_equal_to_boxes():
    """decompose with an explicit cell partition that repeats the boxes
    (ids shifted, one id unused) gives the same subdomains, owners and
    weights as the boxes themselves."""
    import numpy as np
    import workloads as W
    from oracle.mesh import build_mesh
    from oracle.dd import decompose
    w = W.box(7, 5, 4, parts=(3, 2, 2), overlap=1, holes=(((2, 4), (1, 3), (0, 4)),))
    m = build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active)
    ref = decompose(m, w.parts, w.overlap)
    c = np.arange(w.nx * w.ny * w.nz)
    ci, cj, ck = c % w.nx, (c // w.nx) % w.ny, c // (w.nx * w.ny)
    box = (ci * 3 // w.nx) + 3 * ((cj * 2 // w.ny) + 2 * (ck * 2 // w.nz))
    got = decompose(m, (1, 1, 1), w.overlap, cell_part=2 * box + 5)
    assert got.nsub == ref.nsub
    assert np.array_equal(got.box_of_cell, ref.box_of_cell)
    assert np.array_equal(got.owner, ref.owner)
    for i in range(ref.nsub):
        assert np.array_equal(got.N[i], ref.N[i])
        assert np.array_equal(got.D[i], ref.D[i])


def test_classical_pencil_has_too_many_large_eigenvalues():
    """Sec. 3.2, remark on eq. "eigGenEOClassis": without the filter
    (I - xi_0j), the pencil D_j A_j D_j V = lambda A_j^Neu V has many large
    eigenvalues (the gradients of the kept vertices, which A_j^Neu nearly
    annihilates), while the filtered pencil of eq. "eigAtildeBAS" keeps only
    the few that matter (none on this Dirichlet beam with holes)."""
    import numpy as np
    import scipy.linalg as sla
    import workloads as W
    from oracle.mesh import build_mesh
    from oracle.fem import assemble_A, local_element_A
    from oracle.dd import decompose
    from oracle.coarse import local_gevp, tau_paper
    w = W.beam_holes(4, natural_holes=False)
    m = build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active)
    A = assemble_A(m, w)
    AT = local_element_A(m, w)
    dec = decompose(m, w.parts, w.overlap)
    tp = tau_paper(w.tau, "reciprocal")
    j = 1
    g = local_gevp(m, w, A, AT, dec, j)
    D = dec.D[j]
    Ai = g.Ai.toarray() if hasattr(g.Ai, "toarray") else np.asarray(g.Ai)
    classical = sla.eigvalsh(D[:, None] * Ai * D[None, :], np.asarray(g.Aneu))
    n_classical = int((classical > tp).sum())
    n_filtered = int((g.lam > tp).sum())
    assert n_filtered == 0
    assert n_classical > 50
    # they are gradient-driven, far above tau (order 1/gamma)
    assert classical[classical > tp].min() > 100 * tp


def test_curl_route_against_assembled_product_at_small_gamma():
    """Where the two Galerkin routes differ.  For the global gradients G the
    curl-curl part vanishes exactly (K G = 0, Sec. 1: the gradients span the
    kernel of the discrete curl-curl operator), so the exact coarse matrix is
    E = gamma G^T M G.  The assembled product G^T (A G) carries the rounding
    of K G, about u |K|, which relative to gamma |M| grows as 1/gamma; the
    curl route (C G)^T (C G) + gamma G^T M G carries only (u |C|)^2.
    Measured here under a 1e3 contrast of mu^-1: the assembled route loses
    digits in proportion to 1/gamma and turns indefinite at gamma = 1e-12,
    the curl route stays at the rounding level of G^T M G."""
    from oracle.fem import assemble_mass
    from oracle.coarse import galerkin
    errs = []
    for g in (1e-2, 1e-6, 1e-10, 1e-12):
        rng = np.random.default_rng(1)
        w = small(n=(6, 5, 4), gamma=g, mu=10.0 ** rng.uniform(0, 3, 120))
        m, A, AT, dec = setup(w)
        G = gradient_dofs(m)
        Eref = (w.gamma * (G.T @ (assemble_mass(m, w) @ G))).toarray()
        Ec = galerkin(m, w, G)
        Ec = Ec.toarray() if sp.issparse(Ec) else np.asarray(Ec)
        Ea = (G.T @ (A @ G)).toarray()
        nr = np.abs(Eref).max()
        e_curl, e_asm = np.abs(Ec - Eref).max() / nr, np.abs(Ea - Eref).max() / nr
        assert e_curl <= 1e-14
        errs.append(e_asm)
        if g == 1e-12:
            assert np.linalg.eigvalsh(0.5 * (Ea + Ea.T))[0] < 0 < np.linalg.eigvalsh(Ec)[0]
    # the assembled route's error grows at least like 1/gamma (factor 1e4 per
    # 1e-4 of gamma, less a margin of 10)
    assert errs[1] > 1e3 * errs[0] and errs[2] > 1e3 * errs[1]
    assert errs[2] > 1e-3 and errs[3] > 1.0


@pytest.mark.parametrize("case", ["snk_geneo_hole", "paper_tau"])
def test_balanced_start_one_coarse_solve(case):
    """Balanced form of M^-1_AS,2 (closed form at the end of Sec. 3.2): for
    r with Z^T r = 0 the apply w + Z E^-1 Z^T (r - A w) equals the literal
    four-step apply (the first term and (I - P0^T) drop out); PCG from
    x0 = Z E^-1 Z^T b then reaches the direct solution with the literal
    form's iteration count (+-1) and keeps Z^T r small."""
    if case == "snk_geneo_hole":
        w = small(n=(6, 6, 4), parts=(2, 2, 2), overlap=1, gamma=1e-4,
                  holes=[((2, 4), (2, 4), (0, 4))])
        prob = build_problem(w)
    else:
        w = small(n=(6, 5, 4), parts=(2, 2, 1), overlap=1, tau=3.0)
        prob = build_problem(w, tau_convention="paper")
        assert len(prob.geneo) > 0
    A, Z = prob.A, prob.Z
    rng = np.random.default_rng(4)
    rt = rng.standard_normal(A.shape[0])
    # (I - P0^T) r~, so Z^T r = 0 up to the rounding of A Z E^-1 Z^T r~
    # (gamma = 1e-4 makes the gradient part of Z E^-1 Z^T r~ large)
    r = rt - A @ prob.M.coarse(rt)
    assert np.linalg.norm(Z.T @ r) <= 1e-6 * np.linalg.norm(Z.T @ rt)
    lit, bal = prob.M.apply(r), prob.M.apply_balanced(r)
    assert np.linalg.norm(bal - lit) <= 1e-6 * np.linalg.norm(lit)
    x = direct_solve(A, prob.b[0])
    a = solve(prob, tol=1e-12, maxit=500)
    b = solve(prob, tol=1e-12, maxit=500, balanced=True)
    assert b.relres <= 1e-12 and abs(a.iters - b.iters) <= 1
    ea = np.linalg.norm(a.x - x) / np.linalg.norm(x)
    eb = np.linalg.norm(b.x - x) / np.linalg.norm(x)
    assert eb <= 2 * ea + 1e-12
    rb = prob.b[0] - A @ b.x
    assert np.linalg.norm(Z.T @ rb) <= 1e-6 * np.linalg.norm(prob.b[0])


def test_refined_direct_solve_against_high_precision():
    """refined_direct_solve against a 50-digit solve of the same float64 A
    and b (mpmath LU), on a small case made ill conditioned by gamma = 1e-6
    under a 1e3 contrast of mu^-1 (kappa(A) near 2e11): the plain sparse
    solve's forward error is near kappa u (5.6e-7 measured), the refined
    one's near kappa times the extended residual's unit roundoff (2.4e-10
    measured with a 64-bit significand)."""
    mpmath = pytest.importorskip("mpmath")
    from oracle.solver import refined_direct_solve
    rng = np.random.default_rng(2)
    w = small(n=(3, 3, 3), parts=(1, 1, 1), gamma=1e-6, mu=10.0 ** rng.uniform(0, 3, 27))
    m, A, AT, dec = setup(w)
    b = assemble_rhs(m, w)[0]
    mpmath.mp.dps = 50
    xm = mpmath.lu_solve(mpmath.matrix(A.toarray().tolist()), mpmath.matrix(b.tolist()))
    xe = np.array([float(v) for v in xm])
    err = lambda x: np.linalg.norm(x - xe) / np.linalg.norm(xe)
    x1, hist = refined_direct_solve(A, b, steps=3)
    assert err(direct_solve(A, b)) > 1e-8
    assert err(x1) <= 1e-8
    assert hist[-1] <= 1e-8


def test_gmres_right_minimises_the_residual():
    """Right-preconditioned GMRES (Sec. 4's Krylov method): after k steps
    from x0 = 0, x_k minimises ||b - A x|| over the preconditioned Krylov
    space M^-1 K_k(A M^-1, b).  Checked against a dense least-squares solve
    over an explicit basis of that space, for every k up to convergence, and
    the solve reaches the direct solution."""
    from oracle.solver import gmres_right
    w = small(n=(5, 4, 4), parts=(2, 2, 1), overlap=1, gamma=1e-2)
    prob = build_problem(w)
    A = prob.A.toarray()
    b = prob.b[0]
    Minv = np.array([prob.M.apply(e) for e in np.eye(len(b))]).T
    AM = A @ Minv
    for k in (1, 3, 6, 10):
        r = gmres_right(prob.A, b, prob.M.apply, tol=1e-300, maxit=k, restart=50)
        K = np.empty((len(b), k))
        v = b / np.linalg.norm(b)
        for j in range(k):  # orthonormal Krylov basis (two Gram-Schmidt passes)
            for _ in range(2):
                v = v - K[:, :j] @ (K[:, :j].T @ v)
            K[:, j] = v / np.linalg.norm(v)
            v = AM @ K[:, j]
        y, *_ = np.linalg.lstsq(AM @ K, b, rcond=None)
        best = np.linalg.norm(b - AM @ K @ y)
        assert r.iters == k
        assert abs(np.linalg.norm(b - A @ r.x) - best) <= 1e-8 * np.linalg.norm(b)
    r = gmres_right(prob.A, b, prob.M.apply, tol=1e-10)
    x = direct_solve(prob.A, b)
    assert r.relres <= 1e-10
    assert np.linalg.norm(r.x - x) <= 1e-6 * np.linalg.norm(x)
