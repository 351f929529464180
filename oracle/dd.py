"""Overlapping domain decomposition of the oracle (Sec. 2).

* boxes: cell (i,j,k) belongs to box (floor(i px/nx), floor(j py/ny),
  floor(k pz/nz)); boxes without active cells are dropped, the rest keep
  their lexicographic order;
* overlap: L times, add every active cell that shares a vertex with the
  subdomain ("one layer of elements is added in each direction", Sec. 4);
* N_i: interior (non-Dirichlet) edges of the tetrahedra of Omega_i, sorted
  (the restriction R_i of Sec. 2);
* partition of unity (Sec. 2, eq. "PoU"; the paper fixes only D_i >= 0 and
  sum_i R_i^T D_i R_i = I).  Default 'boolean': every edge is owned by the box
  of the lowest-numbered active cell that contains it and D_i(e) = 1 iff i
  owns e.  With this choice the split near-kernel columns of different
  subdomains have disjoint supports, so removing floating components makes Z
  full rank.  Alternative 'core': D_i(e) = chi_i(e) / sum_j chi_j(e) with
  chi_i(e) = 1 iff e in N_i and e lies on no face of the artificial boundary
  of Omega_i (a face with one tetrahedron in Omega_i and two in Omega); its
  split near-kernel columns can be linearly dependent across subdomains;
* k0 (Sec. 2, eq. "k0") and k1 (largest number of subdomains sharing a cell);
* A_i = R_i A R_i^T (Sec. 2, eq. "AS") and A_i^Neu, the form integrated over
  Omega_i only with the global Dirichlet condition kept (Sec. 2).
"""
from __future__ import annotations

from dataclasses import dataclass
import numpy as np
import scipy.sparse as sp

from .fem import assemble_edges, mirror_upper


@dataclass
class Decomposition:
    nsub: int
    box_of_cell: np.ndarray      # [ncells] subdomain id of the box or -1
    sub_cells: list              # per subdomain: sorted active cell ids of Omega_i
    sub_tets: list               # per subdomain: sorted tet ids
    N: list                      # per subdomain: sorted dof ids (R_i)
    core: list                   # per subdomain: bool per local dof (chi_i)
    mult: np.ndarray             # [ndofs] sum_j chi_j(e)
    D: list                      # per subdomain: float64 per local dof
    cell_mult: np.ndarray        # [ncells] number of subdomains containing the cell
    owner: np.ndarray            # [ndofs] owning subdomain (boolean PoU)
    pou: str


def dilate(mask3, active3):
    """One layer: cells sharing a vertex (27-neighbourhood) with the set."""
    nz, ny, nx = mask3.shape
    out = mask3.copy()
    pad = np.pad(mask3, 1)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                out |= pad[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
    return out & active3


def decompose(mesh, parts, overlap, pou="boolean", cell_part=None):
    """Boxes (parts = (px, py, pz)), or any cell partition (cell_part: a
    non-negative id per active cell, as from a graph partitioner; Sec. 4
    uses METIS partitions for its strong scaling study).  Parts that hold
    no active cell are skipped; the others are numbered in increasing id."""
    nx, ny, nz = mesh.nx, mesh.ny, mesh.nz
    px, py, pz = parts
    ncells = nx * ny * nz
    c = np.arange(ncells)
    ci, cj, ck = c % nx, (c // nx) % ny, c // (nx * ny)
    active = np.zeros(ncells, dtype=bool)
    active[mesh.cells] = True
    if cell_part is None:
        bid = (ci * px // nx) + px * ((cj * py // ny) + py * (ck * pz // nz))
        nb = px * py * pz
    else:
        bid = np.where(active, np.asarray(cell_part, dtype=np.int64), 0)
        nb = int(bid[active].max()) + 1
    present = np.unique(bid[active])
    renum = np.full(nb, -1)
    renum[present] = np.arange(len(present))
    box_of_cell = np.where(active, renum[bid], -1)
    nsub = len(present)

    # tet ids of each cell: active cells are numbered by rank, 6 tets each
    cell_rank = np.full(ncells, -1)
    cell_rank[mesh.cells] = np.arange(len(mesh.cells))
    active3 = active.reshape(nz, ny, nx)

    # global face incidence count (1 = physical boundary, 2 = interior)
    gcount = mesh.face_count

    sub_cells, sub_tets, N, core_list = [], [], [], []
    cell_mult = np.zeros(ncells, dtype=np.int64)
    nd = mesh.ndofs
    mult = np.zeros(nd, dtype=np.int64)
    for i in range(nsub):
        m3 = (box_of_cell == i).reshape(nz, ny, nx)
        for _ in range(overlap):
            m3 = dilate(m3, active3)
        cells_i = np.nonzero(m3.reshape(-1))[0]
        cell_mult[cells_i] += 1
        tets_i = (6 * cell_rank[cells_i][:, None] + np.arange(6)[None, :]).reshape(-1)
        tets_i.sort()
        dofs = mesh.edge_dof[mesh.tet_edges[tets_i].reshape(-1)]
        Ni = np.unique(dofs[dofs >= 0])
        # artificial boundary faces of Omega_i
        fids, lc = np.unique(mesh.tet_faces[tets_i].reshape(-1), return_counts=True)
        art = fids[(lc == 1) & (gcount[fids] == 2)]
        f = mesh.faces[art]
        nv = mesh.nverts
        ukeys = mesh.edges[:, 0] * nv + mesh.edges[:, 1]
        fe = np.concatenate([np.searchsorted(ukeys, f[:, 0] * nv + f[:, 1]),
                             np.searchsorted(ukeys, f[:, 0] * nv + f[:, 2]),
                             np.searchsorted(ukeys, f[:, 1] * nv + f[:, 2])])
        art_dofs = mesh.edge_dof[fe]
        art_dofs = np.unique(art_dofs[art_dofs >= 0])
        core = ~np.isin(Ni, art_dofs)
        mult[Ni[core]] += 1
        sub_cells.append(cells_i)
        sub_tets.append(tets_i)
        N.append(Ni)
        core_list.append(core)
    assert np.all(mult >= 1), "every dof must be core in some subdomain"
    # owner: box of the lowest-numbered active cell containing the edge
    first_cell = np.full(len(mesh.edges), np.iinfo(np.int64).max)
    np.minimum.at(first_cell, mesh.tet_edges.reshape(-1), np.repeat(mesh.tet_cell, 6))
    owner = box_of_cell[first_cell[mesh.dof_edge]]
    if pou == "boolean":
        D = [np.where(owner[N[i]] == i, 1.0, 0.0) for i in range(nsub)]
    elif pou == "core":
        D = [np.where(core_list[i], 1.0, 0.0) / mult[N[i]] for i in range(nsub)]
    else:
        raise ValueError(pou)
    return Decomposition(nsub, box_of_cell, sub_cells, sub_tets, N, core_list, mult, D,
                         cell_mult, owner, pou)


def restriction(dec, i, n):
    """R_i as a sparse n_i x n Boolean matrix."""
    Ni = dec.N[i]
    return sp.csr_matrix((np.ones(len(Ni)), (np.arange(len(Ni)), Ni)), shape=(len(Ni), n))


def k0(A, dec):
    """k0 = max_i #{j : R_j A R_i^T != 0} (Sec. 2, eq. "k0"), structurally."""
    n = A.shape[0]
    memb = sp.csr_matrix((np.ones(sum(len(x) for x in dec.N)),
                          (np.concatenate(dec.N),
                           np.concatenate([np.full(len(x), i) for i, x in enumerate(dec.N)]))),
                         shape=(n, dec.nsub))
    P = A.copy()
    P.data = np.ones_like(P.data)
    C = (memb.T @ P @ memb).toarray()
    return int((C != 0).sum(axis=1).max())


def k1(dec):
    """Largest number of subdomains whose intersection has non-zero measure."""
    return int(dec.cell_mult.max())


def local_dirichlet(A, dec, i):
    """A_i = R_i A R_i^T, dense."""
    Ni = dec.N[i]
    return A[Ni][:, Ni].toarray()


def local_neumann(mesh, AT, dec, i):
    """A_i^Neu: element matrices of the tetrahedra of Omega_i only, restricted
    to N_i (Dirichlet dofs of E x n = 0 on the physical boundary removed)."""
    Af = assemble_edges(mesh, AT, tet_subset=dec.sub_tets[i])
    edges = mesh.dof_edge[dec.N[i]]
    An = mirror_upper(Af[edges][:, edges])
    return An.toarray()
