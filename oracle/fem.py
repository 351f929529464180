"""Lowest-order Nedelec (Whitney) discretisation of the positive Maxwell
bilinear form

    a(u, v) = int mu^-1 curl u . curl v + gamma eps u . v      (Sec. 2, eq.
                                                            "bilinearformposmax")

giving A = K + gamma M (Sec. 1, eq. "discretemaxwell") and the load
l(v) = int f . v (Sec. 2).

Whitney basis of edge (a, b) of a tetrahedron, a < b by global vertex id:
W_ab = lambda_a grad lambda_b - lambda_b grad lambda_a, with
curl W_ab = 2 grad lambda_a x grad lambda_b and
int_T lambda_i lambda_j = |T| (1 + delta_ij) / 20.
Coefficients are constant per cubic cell (all six tetrahedra share them).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import LOCAL_EDGES, edge_slot


def barycentric_gradients(P):
    """P: [nt, 4, 3] vertex coordinates.  Returns (grads [nt, 4, 3], vol [nt]).
    x - p0 = sum_k lambda_k (p_k - p0) for k = 1..3, so grad lambda_k is the
    k-th column of J^-1 where J has rows p_k - p0; grad lambda_0 = -sum."""
    J = P[:, 1:, :] - P[:, :1, :]
    Jinv = np.linalg.inv(J)
    g = np.empty_like(P)
    g[:, 1:, :] = np.transpose(Jinv, (0, 2, 1))
    g[:, 0, :] = -g[:, 1:, :].sum(axis=1)
    vol = np.abs(np.linalg.det(J)) / 6.0
    return g, vol


def element_matrices(P, mu_inv, eps):
    """Curl-curl and mass element matrices [nt, 6, 6] on LOCAL_EDGES.
    K_T[e,f] = mu^-1 |T| curlW_e . curlW_f;
    M_T[e,f] = eps int W_e . W_f expanded with int lambda_i lambda_j."""
    g, vol = barycentric_gradients(P)
    nt = P.shape[0]
    curl = np.empty((nt, 6, 3))
    for e, (a, b) in enumerate(LOCAL_EDGES):
        curl[:, e, :] = 2.0 * np.cross(g[:, a, :], g[:, b, :])
    K = (mu_inv * vol)[:, None, None] * np.einsum('tei,tfi->tef', curl, curl)
    GG = np.einsum('tai,tbi->tab', g, g)
    Ml = (vol / 20.0)[:, None, None] * (np.ones((4, 4)) + np.eye(4))[None]
    M = np.empty((nt, 6, 6))
    for e, (a, b) in enumerate(LOCAL_EDGES):
        for f, (c, d) in enumerate(LOCAL_EDGES):
            M[:, e, f] = (Ml[:, a, c] * GG[:, b, d] - Ml[:, a, d] * GG[:, b, c]
                          - Ml[:, b, c] * GG[:, a, d] + Ml[:, b, d] * GG[:, a, c])
    M *= eps[:, None, None]
    return K, M, vol


def tet_coefficients(mesh, w):
    """Per-tetrahedron mu^-1 and eps from the per-cell workload arrays."""
    return w.mu_inv[mesh.tet_cell], w.eps[mesh.tet_cell]


def local_element_A(mesh, w):
    """A_T = K_T + gamma M_T for every tetrahedron."""
    mu, ep = tet_coefficients(mesh, w)
    K, M, _ = element_matrices(mesh.coords[mesh.tets], mu, ep)
    return K + w.gamma * M


def assemble_edges(mesh, AT, tet_subset=None):
    """Sum element matrices over all edges (Dirichlet included), CSR."""
    te = mesh.tet_edges if tet_subset is None else mesh.tet_edges[tet_subset]
    AT = AT if tet_subset is None else AT[tet_subset]
    rows = np.repeat(te, 6, axis=1).reshape(-1)
    cols = np.tile(te, (1, 6)).reshape(-1)
    ne = len(mesh.edges)
    return sp.coo_matrix((AT.reshape(-1), (rows, cols)), shape=(ne, ne)).tocsr()


def mirror_upper(A):
    """Copy the upper triangle onto the lower so A is bit-symmetric."""
    U = sp.triu(A, 0, format='csr')
    S = sp.triu(A, 1, format='csr')
    return (U + S.T).tocsr()


def assemble_A(mesh, w):
    """Global A = K + gamma M over interior (non-Dirichlet) edges; the
    Dirichlet dofs of E x n = 0 are eliminated (rows/cols removed)."""
    Afull = assemble_edges(mesh, local_element_A(mesh, w))
    A = Afull[mesh.dof_edge][:, mesh.dof_edge]
    A = mirror_upper(A)
    A.sort_indices()
    return A


def assemble_K(mesh, w):
    """Curl-curl part only (gamma = 0), interior dofs."""
    mu, ep = tet_coefficients(mesh, w)
    K, _, _ = element_matrices(mesh.coords[mesh.tets], mu, ep)
    Kf = assemble_edges(mesh, K)
    return mirror_upper(Kf[mesh.dof_edge][:, mesh.dof_edge])


def edge_vectors(mesh):
    """t_e = x_head - x_tail."""
    return mesh.coords[mesh.edges[:, 1]] - mesh.coords[mesh.edges[:, 0]]


def assemble_rhs(mesh, w):
    """Load b_e = int f . W_e for f in the Whitney space: f = sum_e c_e W_e
    with c_e = f_e . t_e (exact for constant f), so b = M_1 c with M_1 the
    eps = 1 mass matrix over all edges; rows restricted to interior dofs.
    Returns [nrhs, ndofs]."""
    _, M, _ = element_matrices(mesh.coords[mesh.tets], np.ones(len(mesh.tets)),
                               np.ones(len(mesh.tets)))
    M1 = assemble_edges(mesh, M)
    base, d = edge_slot(mesh)
    t = edge_vectors(mesh)
    out = []
    for r in range(w.nrhs):
        fe = w.f_slot[r][base, d]                  # [nedges, 3]
        c = np.einsum('ei,ei->e', fe, t)
        out.append((M1 @ c)[mesh.dof_edge])
    return np.array(out)


def curl_operator(mesh, w, tet_subset=None):
    """Sparse C (3 ntets x ndofs): row 3T+d holds sqrt(mu^-1_T |T|) times the
    d-th component of curl W_e for the unknowns e of T, so that
    K = C^T C (the curl-curl part of eq. "bilinearformposmax").  Products
    C Z stay accurate for gradient columns: the curl of a gradient is a
    rounding-size vector that enters K-energies squared."""
    g, vol = barycentric_gradients(mesh.coords[mesh.tets])
    mu, _ = tet_coefficients(mesh, w)
    sc = np.sqrt(mu * vol)
    nt = len(mesh.tets)
    rows, cols, vals = [], [], []
    for e, (a, b) in enumerate(LOCAL_EDGES):
        cv = 2.0 * np.cross(g[:, a, :], g[:, b, :]) * sc[:, None]
        dof = mesh.edge_dof[mesh.tet_edges[:, e]]
        ok = dof >= 0
        if tet_subset is not None:
            ok &= tet_subset
        for d in range(3):
            rows.append(3 * np.nonzero(ok)[0] + d)
            cols.append(dof[ok])
            vals.append(cv[ok, d])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(3 * nt, mesh.ndofs))


def assemble_mass(mesh, w):
    """eps-weighted mass matrix over interior dofs (the M of A = K + gamma M)."""
    mu, ep = tet_coefficients(mesh, w)
    _, M, _ = element_matrices(mesh.coords[mesh.tets], mu, ep)
    return mirror_upper(assemble_edges(mesh, M)[mesh.dof_edge][:, mesh.dof_edge])
