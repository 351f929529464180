"""Mesh topology of the oracle: Kuhn tetrahedra on a structured grid of cubic
cells, edges oriented from lower to higher vertex id, Dirichlet boundary by
elimination, and the integer incidence matrices.

Paper: Sec. 4 uses a Cartesian mesh (h = 1/16) and lowest-order Nedelec
edge elements; the Dirichlet condition E x n = 0 of Sec. 1, eq.
"positivemaxwell"; the gradient matrix C / G whose columns span the kernel of
the discrete curl-curl operator (Sec. 1 and the definition "near-kernelCS" of
Sec. 2).
"""
from __future__ import annotations

from dataclasses import dataclass
import numpy as np
import scipy.sparse as sp

# the six Kuhn tetrahedra of a cube: walk from the cell origin along the axes
# in the order of each permutation (lexicographic order of permutations)
PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
# local edges (a, b) of a tetrahedron, a < b; local vertex order is the
# global order because every Kuhn walk step increases the vertex id
LOCAL_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
LOCAL_FACES = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]


@dataclass
class Mesh:
    nx: int
    ny: int
    nz: int
    h: np.ndarray            # (3,) cell sizes
    nverts: int
    coords: np.ndarray       # [nverts, 3]
    cells: np.ndarray        # active cell ids, ascending
    tets: np.ndarray         # [ntets, 4] vertex ids (ascending in each row)
    tet_cell: np.ndarray     # [ntets] cell id
    edges: np.ndarray        # [nedges, 2] (tail, head), tail < head, lexicographic
    tet_edges: np.ndarray    # [ntets, 6] edge ids of LOCAL_EDGES
    faces: np.ndarray        # [nfaces, 3] sorted vertex triples, lexicographic
    tet_faces: np.ndarray    # [ntets, 4]
    face_count: np.ndarray   # [nfaces] number of incident active tets
    dir_edge: np.ndarray     # [nedges] bool: Dirichlet (on a boundary face)
    dir_vert: np.ndarray     # [nverts] bool: Dirichlet vertex
    used_vert: np.ndarray    # [nverts] bool: vertex of an active tet
    edge_dof: np.ndarray     # [nedges] dof id or -1
    dof_edge: np.ndarray     # [ndofs] edge id
    vert_dof: np.ndarray     # [nverts] interior-vertex id or -1
    dof_vert: np.ndarray     # [nvdofs] vertex id

    @property
    def ndofs(self):
        return len(self.dof_edge)

    @property
    def nvdofs(self):
        return len(self.dof_vert)


def vertex_id(i, j, k, nx, ny):
    return i + (nx + 1) * (j + (ny + 1) * k)


def build_mesh(nx, ny, nz, h, active, natural=None):
    """Split every active cell into six Kuhn tetrahedra, number the edges in
    lexicographic (tail, head) order and mark the Dirichlet boundary: faces
    with exactly one incident active tetrahedron carry E x n = 0 (Sec. 1,
    eq. "positivemaxwell"), so their edges and vertices are eliminated from
    the unknowns.

    natural (optional, uint8 per cell): bit 2a + s set marks the face of the
    cell on axis a (x, y, z) at its lower (s = 0) or upper (s = 1) side as a
    natural (Neumann) boundary when it lies on the boundary, as on the hole
    surfaces and lateral faces of Sec. 4; only the remaining boundary faces
    are Dirichlet."""
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (3,)).copy()
    nverts = (nx + 1) * (ny + 1) * (nz + 1)
    v = np.arange(nverts)
    vi = v % (nx + 1)
    vj = (v // (nx + 1)) % (ny + 1)
    vk = v // ((nx + 1) * (ny + 1))
    coords = np.stack([vi * h[0], vj * h[1], vk * h[2]], axis=1)

    active = np.asarray(active).reshape(-1)
    cells = np.nonzero(active)[0].astype(np.int64)
    ci = cells % nx
    cj = (cells // nx) % ny
    ck = cells // (nx * ny)
    v0 = vertex_id(ci, cj, ck, nx, ny)
    stride = [1, nx + 1, (nx + 1) * (ny + 1)]
    tets = np.empty((6 * len(cells), 4), dtype=np.int64)
    for p, (a, b, c) in enumerate(PERMS):
        tets[p::6, 0] = v0
        tets[p::6, 1] = v0 + stride[a]
        tets[p::6, 2] = v0 + stride[a] + stride[b]
        tets[p::6, 3] = v0 + stride[a] + stride[b] + stride[c]
    tet_cell = np.repeat(cells, 6)

    # edges: unique (tail, head) pairs in lexicographic order
    pairs = np.concatenate([tets[:, [a, b]] for a, b in LOCAL_EDGES])
    keys = pairs[:, 0] * nverts + pairs[:, 1]
    ukeys, inv = np.unique(keys, return_inverse=True)
    edges = np.stack([ukeys // nverts, ukeys % nverts], axis=1)
    tet_edges = inv.reshape(6, -1).T.copy()

    # faces: unique sorted triples
    tri = np.concatenate([tets[:, list(f)] for f in LOCAL_FACES])
    fkeys = (tri[:, 0] * nverts + tri[:, 1]) * nverts + tri[:, 2]
    ufk, finv, fcount = np.unique(fkeys, return_inverse=True, return_counts=True)
    faces = np.stack([ufk // (nverts * nverts), (ufk // nverts) % nverts, ufk % nverts], axis=1)
    tet_faces = finv.reshape(4, -1).T.copy()

    bmask = fcount == 1
    if natural is not None:
        # the cell face each boundary triangle lies on, from its one tetrahedron
        ntet = len(tets)
        owner = np.empty(len(faces), dtype=np.int64)
        owner[tet_faces.reshape(-1)] = np.repeat(np.arange(ntet), 4)
        bidx = np.nonzero(bmask)[0]
        cell = tet_cell[owner[bidx]]
        fc = np.stack([vi[faces[bidx]], vj[faces[bidx]], vk[faces[bidx]]], axis=2)  # [nb, 3 v, 3 axes]
        lo = np.stack([cell % nx, (cell // nx) % ny, cell // (nx * ny)], axis=1)
        flat = np.all(fc == fc[:, :1, :], axis=1)       # axes on which the triangle is flat
        assert np.all(flat.sum(1) == 1)
        axis = np.argmax(flat, axis=1)
        side = fc[np.arange(len(bidx)), 0, axis] - lo[np.arange(len(bidx)), axis]
        assert np.all((side == 0) | (side == 1))
        nat = (np.asarray(natural, dtype=np.int64)[cell] >> (2 * axis + side)) & 1
        bmask = bmask.copy()
        bmask[bidx[nat == 1]] = False
    bface = faces[bmask]
    dir_vert = np.zeros(nverts, dtype=bool)
    dir_vert[bface.reshape(-1)] = True
    bpairs = np.concatenate([bface[:, [0, 1]], bface[:, [0, 2]], bface[:, [1, 2]]])
    bkeys = np.unique(bpairs[:, 0] * nverts + bpairs[:, 1])
    dir_edge = np.zeros(len(edges), dtype=bool)
    dir_edge[np.searchsorted(ukeys, bkeys)] = True

    used_vert = np.zeros(nverts, dtype=bool)
    used_vert[tets.reshape(-1)] = True

    edge_dof = np.full(len(edges), -1, dtype=np.int64)
    dof_edge = np.nonzero(~dir_edge)[0]
    edge_dof[dof_edge] = np.arange(len(dof_edge))
    vert_dof = np.full(nverts, -1, dtype=np.int64)
    dof_vert = np.nonzero(used_vert & ~dir_vert)[0]
    vert_dof[dof_vert] = np.arange(len(dof_vert))

    return Mesh(nx, ny, nz, h, nverts, coords, cells, tets, tet_cell, edges, tet_edges,
                faces, tet_faces, fcount, dir_edge, dir_vert, used_vert, edge_dof, dof_edge,
                vert_dof, dof_vert)


def edge_slot(mesh):
    """(lower vertex, direction index) of every edge, for reading the per-slot
    source field of the workloads.  Direction d runs along DIRS[d]."""
    nx, ny = mesh.nx, mesh.ny
    t, hd = mesh.edges[:, 0], mesh.edges[:, 1]
    d = np.stack([hd % (nx + 1) - t % (nx + 1),
                  (hd // (nx + 1)) % (ny + 1) - (t // (nx + 1)) % (ny + 1),
                  hd // ((nx + 1) * (ny + 1)) - t // ((nx + 1) * (ny + 1))], axis=1)
    code = d[:, 0] + 2 * d[:, 1] + 4 * d[:, 2]
    # DIRS order: x, y, z, xy, xz, yz, xyz  -> codes 1, 2, 4, 3, 5, 6, 7
    lut = np.full(8, -1)
    lut[[1, 2, 4, 3, 5, 6, 7]] = np.arange(7)
    return t, lut[code]


def gradient_full(mesh):
    """Signed edge-vertex incidence over ALL edges and vertices: the discrete
    gradient of nodal hat functions, (grad phi_v)_e = phi_v(head) - phi_v(tail)
    (the 'gradient matrix' of Sec. 1)."""
    ne = len(mesh.edges)
    rows = np.concatenate([np.arange(ne), np.arange(ne)])
    cols = np.concatenate([mesh.edges[:, 1], mesh.edges[:, 0]])
    vals = np.concatenate([np.ones(ne, dtype=np.int64), -np.ones(ne, dtype=np.int64)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(ne, mesh.nverts))


def curl_full(mesh):
    """Signed face-edge incidence: the boundary of face (a<b<c) is
    (a,b) + (b,c) - (a,c) with edges oriented low->high."""
    nf = len(mesh.faces)
    nv = mesh.nverts
    ukeys = mesh.edges[:, 0] * nv + mesh.edges[:, 1]
    a, b, c = mesh.faces[:, 0], mesh.faces[:, 1], mesh.faces[:, 2]
    eab = np.searchsorted(ukeys, a * nv + b)
    ebc = np.searchsorted(ukeys, b * nv + c)
    eac = np.searchsorted(ukeys, a * nv + c)
    rows = np.concatenate([np.arange(nf)] * 3)
    cols = np.concatenate([eab, ebc, eac])
    vals = np.concatenate([np.ones(nf, np.int64), np.ones(nf, np.int64), -np.ones(nf, np.int64)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, len(mesh.edges)))


def gradient_dofs(mesh):
    """G restricted to interior edges x interior vertices: the columns are the
    readily available near-kernel of A, the gradients of hat
    functions of vertices that are not on the Dirichlet boundary (Sec. 2,
    definition "near-kernelCS")."""
    full = gradient_full(mesh).tocsc()
    return full[mesh.dof_edge][:, mesh.dof_vert].astype(np.float64).tocsr()
