"""Pins of the warm-start oracle (oracle/mlp.py) against what mathematics fixes:
central finite differences of the loss for the hand-written backward pass,
closed-form values of the subspace loss, and feature values on meshes where
they are known by construction."""
import numpy as np
import pytest

import workloads as W
from oracle import mlp


def _b_orthonormal(B, n, q, rng):
    V = rng.standard_normal((n, q))
    L = np.linalg.cholesky(V.T @ B @ V)
    return V @ np.linalg.inv(L).T


def _spd(n, rng):
    M = rng.standard_normal((n, n))
    return M @ M.T / n + np.eye(n)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    F, V, B = [], [], []
    for n, q in ((23, 3), (31, 8), (17, 0)):
        Bj = _spd(n, rng)
        F.append(rng.uniform(0, 1, (n, mlp.NFEAT)))
        V.append(_b_orthonormal(Bj, n, q, rng) if q else np.zeros((n, 0)))
        B.append(Bj)
    theta = mlp.init_params(3) + 0.01 * rng.standard_normal(mlp.NPARAM)
    L0, g = mlp.loss_and_grad(theta, F, V, B)
    assert np.isfinite(L0)
    for idx in rng.choice(mlp.NPARAM, 40, replace=False):
        h = 1e-6 * max(1.0, abs(theta[idx]))
        tp, tm = theta.copy(), theta.copy()
        tp[idx] += h
        tm[idx] -= h
        fd = (mlp.loss_and_grad(tp, F, V, B)[0] - mlp.loss_and_grad(tm, F, V, B)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-5 * max(1.0, abs(fd))


def test_loss_closed_forms():
    rng = np.random.default_rng(1)
    n = 40
    B = _spd(n, rng)
    V = _b_orthonormal(B, n, 8, rng)
    Q, _ = np.linalg.qr(rng.standard_normal((8, 8)))
    # X inside span(V) with B-orthogonal columns of any length: both terms vanish
    Xs = V @ Q @ np.diag(rng.uniform(0.5, 3.0, 8))
    L, dX = mlp.subdomain_loss(Xs, V, B)
    assert abs(L) < 1e-12 and np.abs(dX).max() < 1e-10
    # X B-orthogonal to V with B-orthogonal columns: the first term is exactly 1
    W8 = _b_orthonormal(B, n, 16, rng)
    L, _ = mlp.subdomain_loss(W8[:, 8:] * 7.0, W8[:, :8], B)
    assert abs(L - 1.0) < 1e-12
    # two equal columns: B-cosine 1 on one pair, counted twice
    X2 = np.column_stack([W8[:, 0], W8[:, 0]] + [W8[:, c] for c in range(2, 8)])
    L, _ = mlp.subdomain_loss(X2, W8[:, 8:], B)
    assert abs(L - (1.0 + 0.1 * 2)) < 1e-12


def _features(w):
    from oracle.mesh import build_mesh
    from oracle.dd import decompose
    m = build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active)
    dec = decompose(m, w.parts, w.overlap)
    return m, dec, [mlp.edge_features(m, w, dec, j) for j in range(dec.nsub)]


def test_features_known_values():
    # uniform mu^-1 = 1e3: f0 = 3/6; one subdomain: no artificial boundary
    w = W.box(4, 3, 2, parts=(1, 1, 1), overlap=1, mu_inv=1e3)
    m, dec, F = _features(w)
    f = F[0]
    assert np.allclose(f[:, 0], 0.5)
    assert np.allclose(f[:, 1], 1.0)
    # axis and diagonal directions: unit vectors with |components| in {0, 1/sqrt2, 1/sqrt3, 1}
    assert np.allclose(np.linalg.norm(f[:, 2:], axis=1), 1.0)
    nz = np.sort(np.unique(np.round(f[:, 2:][f[:, 2:] > 0], 12)))
    assert np.allclose(nz, [1 / np.sqrt(3), 1 / np.sqrt(2), 1.0])


def test_features_distance_to_interface():
    # two boxes along x: edges of the plane x = 2 (the faces Omega_0 shares
    # with the active cells outside it, before overlap) have both vertices at
    # hop distance 0 in the subdomain without overlap
    w = W.box(4, 2, 2, parts=(2, 1, 1), overlap=1)
    m, dec, F = _features(w)
    for j in range(dec.nsub):
        edges = m.edges[m.dof_edge[dec.N[j]]]
        d = F[j][:, 1] * 8
        assert d.min() == 0 and d.max() <= 8
        # distances are integers and differ by at most one along an edge's ends
        assert np.allclose(d, np.round(d))
    # with overlap 1 each subdomain covers 3 of the 4 cell layers; its
    # artificial boundary is the plane x = 3 (j = 0) or x = 1 (j = 1)
    xs = m.coords[:, 0] / w.hx
    e0 = m.edges[m.dof_edge[dec.N[0]]]
    on_plane = (np.isclose(xs[e0[:, 0]], 3)) & (np.isclose(xs[e0[:, 1]], 3))
    assert np.all(F[0][on_plane, 1] == 0)
