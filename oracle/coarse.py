"""Coarse space of the oracle.

* Split near-kernel space V_G = span(R_i^T D_i G_i), G_i = R_i G (Sec. 2,
  definition "near-kernelCS").  One column R_i^T D_i R_i g_v per subdomain i
  and interior vertex v that touches an edge e with D_i(e) > 0 (the support
  of D_i).  Z must have full rank (Sec. 3.2, after eq. "V0GenEOAS"), so
  dependent columns are removed: (a) on every connected component of the
  graph of supp(D_i) edges between interior vertices that has no such edge to
  a Dirichlet vertex ("floating"), the columns sum to zero, and the column of
  the highest vertex id is dropped; (b) a column equal to one of an earlier
  subdomain (same vertex, same support) is dropped.  With the Boolean
  partition of unity the supports of different subdomains are disjoint, (b)
  never applies and the remaining columns are independent.
* xi_0i, the A_i-orthogonal projection onto range(G_i) (Sec. 2, lemma with
  eq. "inverseBw", b_i = (A_i ., .)): xi = G_i S_i^-1 G_i^T A_i with
  S_i = G_i^T A_i G_i; dependent columns of G_i (floating components of the
  N_i edge graph) are dropped the same way.
* the filtered GEVP (Sec. 3.2, GEVP "tauthresholdAS", eq. "eigAtildeBAS"):
  (I - xi^T) D_j A_j D_j (I - xi) V = lambda A_j^Neu V, selecting lambda > tau
  and adding the vectors R_j^T D_j (I - xi) V (dense generalized eigensolve).
* Z = [Z_G | Z_GenEO] (eq. "V0GenEOAS") and E = Z^T A Z (Sec. 2).  V_0 is
  the vector-space sum V_G + V_GenEO and Z must be a full-rank basis of it, so
  a GenEO column that lies (numerically) in the span of the SNK columns and
  of the GenEO columns kept before it is dropped: with E_HH - E_HG E_GG^-1
  E_GH the Schur complement of the GenEO block, an ordered Cholesky drops
  column k when its pivot is below DEP_TOL * E_kk.
"""
from __future__ import annotations

from dataclasses import dataclass
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .dd import local_dirichlet, local_neumann


def _components(nodes, a, b):
    """Connected components of the graph on `nodes` with edges (a[k], b[k]).
    Returns dict node -> root (a representative)."""
    parent = {int(v): int(v) for v in nodes}

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for u, v in zip(a.tolist(), b.tolist()):
        ru, rv = find(u), find(v)
        if ru != rv:
            parent[max(ru, rv)] = min(ru, rv)
    return {v: find(v) for v in parent}


def _kept_vertices(mesh, edge_dofs):
    """Interior vertices touched by the given dof edges, minus the highest
    vertex of every component (through those edges, between interior
    vertices) that has no edge to a Dirichlet vertex.  Sorted."""
    ed = mesh.dof_edge[edge_dofs]
    t, h = mesh.edges[ed, 0], mesh.edges[ed, 1]
    it, ih = mesh.vert_dof[t] >= 0, mesh.vert_dof[h] >= 0
    verts = np.unique(np.concatenate([t[it], h[ih]]))
    both = it & ih
    comp = _components(verts, t[both], h[both])
    anchored = set()
    for u, iu, w, iw in zip(t.tolist(), it.tolist(), h.tolist(), ih.tolist()):
        if iu and not iw:
            anchored.add(comp[u])
        if iw and not iu:
            anchored.add(comp[w])
    top = {}
    for v in verts.tolist():
        r = comp[v]
        if r not in anchored:
            top[r] = max(top.get(r, -1), v)
    drop = set(top.values())
    return np.array([v for v in verts.tolist() if v not in drop], dtype=np.int64)


def snk_columns(mesh, dec):
    """List of (subdomain i, vertex v, dof rows, values) of Z_G in column
    order (i ascending, then v ascending), duplicates and floating columns
    removed."""
    cols = []
    seen = set()
    for i in range(dec.nsub):
        Ni, Di = dec.N[i], dec.D[i]
        sup = Di > 0
        cdofs = Ni[sup]
        cvals = Di[sup]
        kept = _kept_vertices(mesh, cdofs)
        ed = mesh.dof_edge[cdofs]
        t, h = mesh.edges[ed, 0], mesh.edges[ed, 1]
        for v in kept.tolist():
            sel_h = h == v
            sel_t = t == v
            rows = np.concatenate([cdofs[sel_h], cdofs[sel_t]])
            vals = np.concatenate([cvals[sel_h], -cvals[sel_t]])
            order = np.argsort(rows)
            rows, vals = rows[order], vals[order]
            key = (v, tuple(rows.tolist()))
            if key in seen:
                continue
            seen.add(key)
            cols.append((i, v, rows, vals))
    return cols


def nk_columns(mesh):
    """Global near-kernel G (coarse variant 'NK' of Sec. 4): one column per
    interior vertex, except the highest vertex of every connected component
    of unknown edges that has no edge to a Dirichlet vertex (possible when
    every boundary face of a component is natural): there G times the
    constant vanishes, and Sec. 3.2 needs a Z of full column rank."""
    G = mesh_gradient(mesh).tocsc()
    kept = set(_kept_vertices(mesh, np.arange(mesh.dof_edge.shape[0])).tolist())
    cols = []
    for k, v in enumerate(mesh.dof_vert.tolist()):
        if v not in kept:
            continue
        s = slice(G.indptr[k], G.indptr[k + 1])
        cols.append((-1, v, G.indices[s].copy(), G.data[s].copy()))
    return cols


def mesh_gradient(mesh):
    from .mesh import gradient_dofs
    return gradient_dofs(mesh)


def local_gradient(mesh, dec, i):
    """G_i = R_i G on the kept (independent) interior vertices of Omega_i;
    dense n_i x m_i with entries +-1.  Returns (G_i, kept vertex ids)."""
    Ni = dec.N[i]
    kept = _kept_vertices(mesh, Ni)
    col = {v: k for k, v in enumerate(kept.tolist())}
    Gi = np.zeros((len(Ni), len(kept)))
    ed = mesh.dof_edge[Ni]
    for r, (t, h) in enumerate(mesh.edges[ed].tolist()):
        if h in col:
            Gi[r, col[h]] += 1.0
        if t in col:
            Gi[r, col[t]] -= 1.0
    return Gi, kept


@dataclass
class LocalGEVP:
    lam: np.ndarray       # all eigenvalues, descending
    V: np.ndarray         # B-orthonormal eigenvectors (columns), same order
    Ai: np.ndarray
    Aneu: np.ndarray
    Gi: np.ndarray
    xi: np.ndarray
    L: np.ndarray


def xi_projector(Ai, Gi):
    """xi_0i = G_i (G_i^T A_i G_i)^-1 G_i^T A_i (A_i-orthogonal projection on
    range G_i parallel to its A_i-orthogonal complement)."""
    if Gi.shape[1] == 0:
        return np.zeros_like(Ai)
    S = Gi.T @ Ai @ Gi
    return Gi @ sla.solve(S, Gi.T @ Ai, assume_a='pos')


def xi_projector_curl(mesh, w, dec, i, Gi):
    """xi_0i with G_i^T A_i formed through the curl operator:
    G_i^T A_i = (C R_i^T G_i)^T (C R_i^T) + gamma G_i^T M_i, which equals the
    assembled product but keeps its small (order gamma) entries accurate."""
    from .fem import curl_operator, assemble_mass
    if Gi.shape[1] == 0:
        return np.zeros((len(dec.N[i]), len(dec.N[i])))
    Ni = dec.N[i]
    Ci = curl_operator(mesh, w)[:, Ni]
    Mi = assemble_mass(mesh, w)[Ni][:, Ni]
    CG = Ci @ Gi
    GtA = (Ci.T @ CG).T + w.gamma * (Mi @ Gi).T
    S = GtA @ Gi
    S = 0.5 * (S + S.T)
    return Gi @ sla.solve(S, GtA, assume_a='pos')


def local_gevp(mesh, w, A, AT, dec, j, pencil="filtered"):
    """Dense solve of GEVP "tauthresholdAS" (eq. "eigAtildeBAS") on Omega_j;
    pencil="classical" solves the unfiltered GEVP of the remark in Sec. 3.2,
    eq. "eigGenEOClassis": D_j A_j D_j V = lambda A_j^Neu V."""
    Ai = local_dirichlet(A, dec, j)
    Aneu = local_neumann(mesh, AT, dec, j)
    Gi, _ = local_gradient(mesh, dec, j)
    Dj = dec.D[j]
    if pencil == "classical":
        xi = np.zeros((len(Ai), len(Ai)))
        Ixi = np.eye(len(Ai))
    elif pencil == "filtered":
        xi = xi_projector_curl(mesh, w, dec, j, Gi)
        Ixi = np.eye(len(Ai)) - xi
    else:
        raise ValueError(pencil)
    L = Ixi.T @ (Dj[:, None] * Ai * Dj[None, :]) @ Ixi
    L = 0.5 * (L + L.T)
    lam, V = sla.eigh(L, Aneu)
    order = np.argsort(lam)[::-1]
    lam, V = lam[order], V[:, order]
    # deterministic sign: largest-magnitude entry positive
    idx = np.argmax(np.abs(V), axis=0)
    sgn = np.sign(V[idx, np.arange(V.shape[1])])
    sgn[sgn == 0] = 1.0
    V = V * sgn[None, :]
    return LocalGEVP(lam, V, Ai, Aneu, Gi, xi, L)


def tau_paper(tau, convention="reciprocal"):
    """Threshold applied to the eigenvalues of eq. "eigAtildeBAS".  The
    paper's experiments select lambda > 10 (Sec. 4).  'reciprocal' reads the
    user tau as the classical-GenEO threshold on the reciprocal pencil, i.e.
    lambda > 1/tau; 'paper' applies tau literally."""
    if convention == "reciprocal":
        return 1.0 / tau
    if convention == "paper":
        return tau
    raise ValueError(convention)


def geneo_columns(mesh, w, A, AT, dec, tau_p, gevps=None, pencil="filtered"):
    """Columns R_j^T D_j (I - xi_0j) V_jk for lambda_jk > tau_p, per subdomain
    in descending lambda order (R_j^T D_j V_jk for the classical pencil, whose
    xi is zero).  Returns (cols, gevps)."""
    cols = []
    out = []
    for j in range(dec.nsub):
        g = gevps[j] if gevps is not None else local_gevp(mesh, w, A, AT, dec, j, pencil)
        out.append(g)
        sel = np.nonzero(g.lam > tau_p)[0]
        Ixi = np.eye(len(g.Ai)) - g.xi
        for k in sel.tolist():
            vec = dec.D[j] * (Ixi @ g.V[:, k])
            cols.append((j, k, dec.N[j].copy(), vec))
    return cols, out


def assemble_Z(n, cols):
    """Sparse n x n0 coarse basis from column lists."""
    rows = np.concatenate([c[2] for c in cols]) if cols else np.zeros(0, np.int64)
    vals = np.concatenate([c[3] for c in cols]) if cols else np.zeros(0)
    cidx = np.concatenate([np.full(len(c[2]), k) for k, c in enumerate(cols)]) if cols \
        else np.zeros(0, np.int64)
    return sp.csc_matrix((vals, (rows, cidx)), shape=(n, len(cols)))


DEP_TOL = 1e-8


def galerkin(mesh, w, X, Y=None):
    """X^T A Y summed element by element, K-part through the curl operator:
    (C X)^T (C Y) + gamma X^T M Y.  Equal to X^T A Y; for gradient-like
    columns it avoids the cancellation of K G = 0 inside assembled A."""
    from .fem import curl_operator, assemble_mass
    Y = X if Y is None else Y
    Cm = curl_operator(mesh, w)
    M = assemble_mass(mesh, w)
    CX, CY = Cm @ X, Cm @ Y
    out = CX.T @ CY + w.gamma * (X.T @ (M @ Y))
    return out


def coarse_matrix(mesh, w, Z, dense_limit=6000):
    """E = Z^T A Z (Sec. 2), element by element (see galerkin); dense below
    dense_limit columns, sparse CSR above."""
    E = galerkin(mesh, w, Z)
    if sp.issparse(E):
        E = sp.csr_matrix(0.5 * (E + E.T))
        return E.toarray() if E.shape[0] <= dense_limit else E
    E = np.asarray(E)
    return 0.5 * (E + E.T)


def independent_geneo(E, n_snk):
    """Indices (relative to the GenEO block) of the GenEO columns kept by
    the ordered Cholesky of the Schur complement of the GenEO block of E
    (pivot >= DEP_TOL * diagonal).  E covers [SNK | GenEO candidates]."""
    m = E.shape[0] - n_snk
    if m == 0:
        return np.zeros(0, np.int64)
    dense = lambda X: X.toarray() if sp.issparse(X) else np.asarray(X)
    Ehh = dense(E[n_snk:, n_snk:])
    diag = np.diag(Ehh).copy()
    if n_snk > 0:
        Egg = E[:n_snk, :n_snk]
        Egh = dense(E[:n_snk, n_snk:])
        if not sp.issparse(Egg):
            S = Ehh - Egh.T @ sla.cho_solve(sla.cho_factor(Egg), Egh)
        else:
            import scipy.sparse.linalg as spla
            S = Ehh - Egh.T @ spla.splu(sp.csc_matrix(Egg)).solve(Egh)
    else:
        S = Ehh
    S = 0.5 * (S + S.T)
    keep = []
    L = np.zeros((m, m))
    for k in range(m):
        piv = S[k, k] - L[k, keep] @ L[k, keep]
        if piv < DEP_TOL * diag[k]:
            continue
        d = np.sqrt(piv)
        L[k, k] = d
        rest = np.arange(k + 1, m)
        L[rest, k] = (S[rest, k] - L[np.ix_(rest, keep)] @ L[k, keep]) / d
        keep.append(k)
    return np.array(keep, dtype=np.int64)
