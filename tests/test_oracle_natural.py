"""Natural (Neumann) boundary faces in the oracle (Sec. 4, mixed boundary
conditions), pinned by what the mathematics and the paper fix:
* with every boundary face natural, every edge is an unknown and no vertex
  is eliminated (the closed-form edge count of the box);
* a natural mark on a face that is not on the boundary changes nothing;
* K G = 0 still holds with the gradients of the vertices on natural faces;
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
