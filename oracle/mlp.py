"""Oracle of the learned warm start for the local eigensolves (float64).

TEST INFRASTRUCTURE ONLY (see the package header).

The method's local generalised eigenproblems (Sec. 3.2, GEVP
"tauthresholdAS") are solved iteratively on the GPU; a small network proposes
the initial block.  Everything here restates that network in plain NumPy:

* per local edge e of subdomain j, five features
    f0 = mean of log10(mu^-1) over the tetrahedra of Omega_j containing e, / 6
    f1 = min(d(tail), d(head), 8) / 8, d = hop distance, along the edges of
         Omega_j's tetrahedra, to the artificial boundary of Omega_j (the
         vertices of Omega_j shared with an active cell outside Omega_j);
         8 when Omega_j has no artificial boundary
    f2..f4 = |x_head - x_tail| / ||x_head - x_tail||, componentwise
* the network 5 -> 128 -> 128 -> 8 with ReLU, parameters flattened as
  W1[128][5], b1[128], W2[128][128], b2[128], W3[8][128], b3[8];
* the training loss of one subdomain, X = network output on its edges
  (n_j x 8), V its locked eigenvectors (B-orthonormal, q_j <= 8 columns),
  B = A_j^Neu (the right-hand operator of the GEVP), G = X^T B X:
    L_j = ||(I - V V^T B) X||_F^2 / ||X||_F^2
          + 0.1 sum_{a != b} G_ab^2 / (G_aa G_bb),
  (the subspace term and the B-cosines between the columns; both are
  invariant to the scale of B, which spans orders of magnitude with mu^-1),
  averaged over the subdomains with q_j > 0, and its gradient by hand.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 128
NOUT = 8
NFEAT = 5
SHAPES = [("W1", (HIDDEN, NFEAT)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)),
          ("b2", (HIDDEN,)), ("W3", (NOUT, HIDDEN)), ("b3", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shp)
        o += k
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1)
                           for name, _ in SHAPES])


def forward(theta, F):
    """F: [n, 5] features -> (out [n, 8], cache)."""
    p = unpack(theta)
    z1 = F @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    out = h2 @ p["W3"].T + p["b3"]
    return out, (F, z1, h1, z2, h2, p)


def backward(cache, dout):
    """Gradient of sum(out * dout) with respect to the flattened parameters."""
    F, z1, h1, z2, h2, p = cache
    g = {}
    g["W3"] = dout.T @ h2
    g["b3"] = dout.sum(axis=0)
    dz2 = (dout @ p["W3"]) * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * (z1 > 0)
    g["W1"] = dz1.T @ F
    g["b1"] = dz1.sum(axis=0)
    return pack(g)


def subdomain_loss(X, V, B):
    """L_j and dL_j/dX for X [n, 8], V [n, q] (V^T B V = I), B [n, n]."""
    BX = B @ X
    nX = float((X * X).sum())
    Gvx = V.T @ BX
    R = X - V @ Gvx
    L1 = float((R * R).sum()) / nX
    G = X.T @ BX
    d = np.diag(G).copy()
    off = ~np.eye(len(d), dtype=bool)
    dd = np.outer(d, d)
    L2 = 0.1 * float((G[off] ** 2 / dd[off]).sum())
    # dL2/dG: off-diagonal 0.2 G_ab / (d_a d_b); diagonal from d_a
    H = np.where(off, 0.2 * G / dd, 0.0)
    H[np.diag_indices(len(d))] = -0.2 * np.where(off, G ** 2 / (dd * d[:, None]), 0.0).sum(1)
    BV = B @ V
    dX = 2.0 * (R - BV @ (V.T @ R)) / nX - 2.0 * L1 * X / nX + 2.0 * BX @ H
    return L1 + L2, dX


def loss_and_grad(theta, F_list, V_list, B_list):
    """Mean loss over subdomains with eigenvectors and its parameter gradient.
    F_list[j]: [n_j, 5]; V_list[j]: [n_j, q_j]; B_list[j]: [n_j, n_j]."""
    use = [j for j in range(len(F_list)) if V_list[j].shape[1] > 0]
    J = len(use)
    total, grad = 0.0, np.zeros(NPARAM)
    for j in use:
        out, cache = forward(theta, F_list[j])
        L, dX = subdomain_loss(out, V_list[j], B_list[j])
        total += L / J
        grad += backward(cache, dX / J)
    return total, grad


def init_params(seed):
    """He-normal weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in SHAPES:
        if name.startswith("W"):
            p[name] = rng.standard_normal(shp) * np.sqrt(2.0 / shp[1])
        else:
            p[name] = np.zeros(shp)
    return pack(p)


def edge_features(mesh, w, dec, j):
    """[n_j, 5] features of the local edges of subdomain j (rows in N_j order)."""
    Nj = dec.N[j]
    edges = mesh.edges[mesh.dof_edge[Nj]]
    tets = dec.sub_tets[j]
    # f0: mean log10 mu^-1 over the tetrahedra of Omega_j containing the edge
    logmu = np.log10(np.asarray(w.mu_inv, dtype=np.float64))
    row_of_edge = {int(e): r for r, e in enumerate(mesh.dof_edge[Nj].tolist())}
    acc = np.zeros(len(Nj))
    cnt = np.zeros(len(Nj))
    for t in tets.tolist():
        lm = logmu[mesh.tet_cell[t]]
        for e in mesh.tet_edges[t].tolist():
            r = row_of_edge.get(int(e))
            if r is not None:
                acc[r] += lm
                cnt[r] += 1
    f0 = acc / np.maximum(cnt, 1) / 6.0
    # f1: hop distance to the artificial boundary
    verts = np.unique(mesh.tets[tets].reshape(-1))
    in_sub = np.zeros(mesh.nx * mesh.ny * mesh.nz, dtype=bool)
    in_sub[dec.sub_cells[j]] = True
    act = np.zeros_like(in_sub)
    act[mesh.cells] = True
    outside = act & ~in_sub
    src = set()
    for v in verts.tolist():
        vi = v % (mesh.nx + 1)
        vj = (v // (mesh.nx + 1)) % (mesh.ny + 1)
        vk = v // ((mesh.nx + 1) * (mesh.ny + 1))
        for dk in (-1, 0):
            for dj in (-1, 0):
                for di in (-1, 0):
                    ci, cj, ck = vi + di, vj + dj, vk + dk
                    if 0 <= ci < mesh.nx and 0 <= cj < mesh.ny and 0 <= ck < mesh.nz:
                        if outside[ci + mesh.nx * (cj + mesh.ny * ck)]:
                            src.add(v)
    adj = {}
    for t in tets.tolist():
        for e in mesh.tet_edges[t].tolist():
            a, b = (int(x) for x in mesh.edges[e])
            adj.setdefault(a, set()).add(b)
            adj.setdefault(b, set()).add(a)
    dist = {v: 8 for v in verts.tolist()}
    frontier = sorted(src)
    for v in frontier:
        dist[v] = 0
    d = 0
    seen = set(frontier)
    while frontier and d < 8:
        d += 1
        nxt = []
        for v in frontier:
            for u in adj.get(v, ()):
                if u not in seen:
                    seen.add(u)
                    dist[u] = d
                    nxt.append(u)
        frontier = nxt
    f1 = np.array([min(dist[int(a)], dist[int(b)], 8) for a, b in edges], dtype=np.float64) / 8.0
    # f2..f4: unit direction, absolute components
    vec = mesh.coords[edges[:, 1]] - mesh.coords[edges[:, 0]]
    u = np.abs(vec) / np.linalg.norm(vec, axis=1, keepdims=True)
    return np.column_stack([f0, f1, u])
