"""Natural (Neumann) boundary faces in the oracle (Sec. 4, mixed boundary
conditions), pinned by what the mathematics and the paper fix:
* with every boundary face natural, every edge is an unknown and no vertex
  is eliminated (the closed-form edge count of the box);
* a natural mark on a face that is not on the boundary changes nothing;
* K G = 0 still holds with the gradients of the vertices on natural faces;
* a manufactured curl-free field whose tangential trace vanishes only on
  the Dirichlet faces is recovered at the expected rate, and not at all
  when the natural faces are made Dirichlet;
* Sec. 4, beam with holes: with Dirichlet conditions on the hole surfaces
  GenEO selects nothing, and with Neumann conditions there it selects
  vectors in every box, the same number in every interior box whatever the
  number of boxes (the paper's count grows as 3(N - 2))."""
import numpy as np
import pytest

import workloads as W
from oracle.mesh import build_mesh


def test_all_natural_box():
    from test_oracle_mesh_fem import box_edges_closed_form
    nx, ny, nz = 4, 3, 2
    nat = np.full(nx * ny * nz, 63, np.uint8)
    m = build_mesh(nx, ny, nz, 1.0, np.ones(nx * ny * nz, np.uint8), natural=nat)
    assert m.ndofs == len(m.edges) == box_edges_closed_form(nx, ny, nz)
    assert not m.dir_vert.any() and m.nvdofs == (nx + 1) * (ny + 1) * (nz + 1)


def test_natural_marks_inside_change_nothing():
    w = W.box(5, 4, 3, parts=(1, 1, 1), holes=(((1, 3), (1, 2), (0, 3)),))
    m0 = build_mesh(w.nx, w.ny, w.nz, 1.0, w.active)
    # mark every face that has an active neighbour (never a boundary face)
    nat = np.zeros(w.nx * w.ny * w.nz, np.uint8)
    act = w.active.reshape(w.nz, w.ny, w.nx).astype(bool)
    for k in range(w.nz):
        for j in range(w.ny):
            for i in range(w.nx):
                for a, (di, dj, dk) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
                    for s, sg in ((0, -1), (1, 1)):
                        ii, jj, kk = i + sg * di, j + sg * dj, k + sg * dk
                        if 0 <= ii < w.nx and 0 <= jj < w.ny and 0 <= kk < w.nz and act[kk, jj, ii]:
                            nat[i + w.nx * (j + w.ny * k)] |= 1 << (2 * a + s)
    m1 = build_mesh(w.nx, w.ny, w.nz, 1.0, w.active, natural=nat)
    assert np.array_equal(m0.dir_edge, m1.dir_edge) and np.array_equal(m0.dir_vert, m1.dir_vert)
    # and the generator marks nothing on a box without holes unless asked
    assert not W.natural_faces(W.box(3, 3, 3), holes=True).any()


def test_curl_kills_gradients_with_natural_faces():
    from oracle.fem import assemble_K
    from oracle.mesh import gradient_dofs
    w = W.beam_holes(4)
    m = build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active, natural=w.natural)
    md = build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active)
    assert m.nvdofs > md.nvdofs  # vertices on the hole surfaces became unknowns
    K = assemble_K(m, w)
    G = gradient_dofs(m)
    assert G.shape == (m.ndofs, m.nvdofs)
    assert abs(K @ G).max() <= 1e-12 * abs(K).max()


@pytest.mark.slow
def test_geneo_needs_natural_holes():
    from oracle.pipeline import build_problem
    counts = {}
    for nsub in (4, 6):
        p = build_problem(W.beam_holes(nsub, natural_holes=True))
        counts[nsub] = [int((g.lam > p.tau_p).sum()) for g in p.gevps]
    pd = build_problem(W.beam_holes(4, natural_holes=False))
    assert all(int((g.lam > pd.tau_p).sum()) == 0 for g in pd.gevps)
    for nsub, c in counts.items():
        assert all(x > 0 for x in c)
        assert len(set(c[1:-1])) == 1       # the same count in every interior box
    assert counts[4][1] == counts[6][1]
    assert counts[4][0] == counts[6][0] and counts[4][-1] == counts[6][-1]


def _natural_error(n, natural=True):
    """Relative discrete L2 error of the FE solution against the edge
    interpolant of E* = grad(sin pi x cos pi y sin pi z) on the unit cube,
    with f = gamma E* (curl E* = 0, so curl E* x n = 0 holds on every face),
    E* x n = 0 on the faces x = 0, 1 and z = 0, 1, and a nonzero tangential
    trace on y = 0, 1, which are the natural faces."""
    import scipy.sparse.linalg as spla
    from oracle.mesh import edge_slot
    from oracle.fem import assemble_A, assemble_rhs, element_matrices, assemble_edges
    from test_oracle_mesh_fem import edge_vectors
    w = W.box(n, n, n, gamma=1.0)
    nat = W.natural_faces(w, sides=((1, 0), (1, 1))) if natural else None
    m = build_mesh(n, n, n, 1.0 / n, w.active, natural=nat)
    pi = np.pi
    Es = lambda x: np.stack([pi * np.cos(pi * x[:, 0]) * np.cos(pi * x[:, 1]) * np.sin(pi * x[:, 2]),
                             -pi * np.sin(pi * x[:, 0]) * np.sin(pi * x[:, 1]) * np.sin(pi * x[:, 2]),
                             pi * np.sin(pi * x[:, 0]) * np.cos(pi * x[:, 1]) * np.cos(pi * x[:, 2])],
                            axis=1)
    base, d = edge_slot(m)
    mid = 0.5 * (m.coords[m.edges[:, 0]] + m.coords[m.edges[:, 1]])
    f_slot = np.zeros((1, m.nverts, 7, 3))
    f_slot[0, base, d] = Es(mid)
    w.f_slot = f_slot
    u = spla.spsolve(assemble_A(m, w).tocsc(), assemble_rhs(m, w)[0])
    t = edge_vectors(m)
    gp = [(0.5 - np.sqrt(15) / 10, 5 / 18), (0.5, 8 / 18), (0.5 + np.sqrt(15) / 10, 5 / 18)]
    pi_u = sum(wq * np.einsum('ei,ei->e', Es(m.coords[m.edges[:, 0]] + s * t), t) for s, wq in gp)
    pi_u = pi_u[m.dof_edge]
    _, M, _ = element_matrices(m.coords[m.tets], np.ones(len(m.tets)), np.ones(len(m.tets)))
    Mf = assemble_edges(m, M)[m.dof_edge][:, m.dof_edge]
    e = u - pi_u
    return np.sqrt(e @ (Mf @ e) / (pi_u @ (Mf @ pi_u)))


@pytest.mark.slow
def test_natural_faces_manufactured_rate():
    errs = [_natural_error(n) for n in (4, 8, 16)]
    rates = [np.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(r >= 0.9 for r in rates), (errs, rates)
    # the same field with Dirichlet y faces is not a solution: no convergence
    assert _natural_error(16, natural=False) > 0.2
