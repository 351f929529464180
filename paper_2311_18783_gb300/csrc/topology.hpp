// Host-side integer topology of the structured Kuhn mesh and of the
// overlapping box decomposition.  Everything here is exact integer work done
// once in set-up; the numerical set-up and the solve run on the GPU.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace geneo {

// seven positive edge directions, in the order of the public slot layout
// (x, y, z, x+y, x+z, y+z, x+y+z)
extern const int kDir[7][3];

struct Topology {
  int nx = 0, ny = 0, nz = 0;
  double h[3] = {0, 0, 0};
  int64_t nverts = 0, ncells = 0;
  std::vector<int32_t> cells;      // active cell ids, ascending
  std::vector<int32_t> cell_rank;  // [ncells] rank among active cells or -1
  std::vector<int32_t> tets;       // [ntets][4] ascending vertex ids
  std::vector<int32_t> tet_cell;   // [ntets]
  std::vector<int32_t> edges;      // [nedges][2] tail, head (lexicographic)
  std::vector<int32_t> edge_dir;   // [nedges] direction index into kDir
  std::vector<int32_t> tet_edges;  // [ntets][6] local pairs (01,02,03,12,13,23)
  std::vector<uint8_t> dir_edge, dir_vert, used_vert;
  std::vector<int32_t> edge_dof, dof_edge, vert_dof, dof_vert;
  std::vector<int32_t> first_cell; // [nedges] lowest active cell containing the edge
  // CSR pattern of A over unknowns
  std::vector<int32_t> rowptr, col;
  // assembly gather lists: nonzero k of A sums element entries
  // cidx[cptr[k] .. cptr[k+1]) = tet*36 + a*6 + b, in tet order
  std::vector<int64_t> cptr;
  std::vector<int32_t> cidx;
  // load gather lists: unknown e sums rows (tet*6 + a), in tet order
  std::vector<int64_t> rptr;
  std::vector<int32_t> ridx;

  int64_t ntets() const { return (int64_t)tet_cell.size(); }
  int64_t nedges() const { return (int64_t)edge_dir.size(); }
  int64_t ndofs() const { return (int64_t)dof_edge.size(); }
  int64_t nnz() const { return (int64_t)col.size(); }
};

struct Decomposition {
  int nsub = 0;
  int overlap = 0;
  std::vector<int32_t> box_of_cell;              // [ncells] or -1
  std::vector<std::vector<int32_t>> sub_cells;   // ascending
  std::vector<int64_t> N_off;                    // [nsub+1]
  std::vector<int32_t> N_idx;                    // concatenated sorted dof ids
  std::vector<int32_t> owner;                    // [ndofs]
  std::vector<int32_t> cell_mult;                // [ncells]
  int k0 = 0, k1 = 0;
  int64_t ni(int i) const { return N_off[i + 1] - N_off[i]; }
};

// Local sparse structure of one subdomain's Dirichlet matrix A_i = R_i A R_i^T
// (same pattern holds A_i^Neu) plus the gather lists of A_i^Neu, which sums
// only the element entries of tetrahedra inside Omega_i.
struct LocalStructure {
  // all subdomains concatenated; rows indexed by the global local-slot number
  std::vector<int64_t> lrowptr;   // [sum_ni + 1]
  std::vector<int32_t> lcol;      // local column index
  std::vector<int32_t> lpos;      // position of the entry in A's CSR
  std::vector<int64_t> ncptr;     // [lnnz + 1] A^Neu gather lists
  std::vector<int32_t> ncidx;     //   tet*36 + a*6 + b
  // prolongation: for each unknown, the local slots that hold it
  std::vector<int64_t> g2l_ptr;   // [n + 1]
  std::vector<int64_t> g2l_slot;  // local slot numbers (global numbering over sum_ni)
  // gradient structure for xi_0i: kept interior vertices of each subdomain
  std::vector<int64_t> xv_off;    // [nsub + 1] offsets into xv_vert
  std::vector<int32_t> xv_vert;   // kept vertex ids (ascending per subdomain)
  std::vector<int32_t> gi_head;   // [sum_ni] local kept-vertex index of head or -1
  std::vector<int32_t> gi_tail;   // [sum_ni] local kept-vertex index of tail or -1
  // vertex stars for S_i = G_i^T A_i G_i: for each kept vertex, local rows with sign
  std::vector<int64_t> star_ptr;  // [total kept + 1]
  std::vector<int32_t> star_row;  // local row (within the subdomain)
  std::vector<int8_t> star_sgn;   // +1 head, -1 tail
};

// Split near-kernel columns R_i^T D_i R_i g_v with the Boolean partition of
// unity (D_i = 1 on unknowns owned by i), floating components removed.
struct SNKColumns {
  std::vector<int32_t> sub, vert;   // per column
  std::vector<int64_t> ptr;         // CSC column pointers
  std::vector<int32_t> row;         // unknown ids
  std::vector<int8_t> sgn;          // +1 / -1
};

// natural (optional): per cell, bit 2a + s marks its face on axis a at side
// s (0 lower, 1 upper) as a natural boundary when that face is on the
// boundary; the other boundary faces are Dirichlet (E x n = 0).
void build_topology(int nx, int ny, int nz, const double h[3], const uint8_t *active,
                    Topology &t, const uint8_t *natural = nullptr);
// Boxes px x py x pz, or (cell_part non-null) the given subdomain of every
// active cell; empty parts are dropped and the rest renumbered in order.
void build_decomposition(const Topology &t, int px, int py, int pz, int overlap,
                         Decomposition &d, const int32_t *cell_part = nullptr);
void build_local_structure(const Topology &t, const Decomposition &d, LocalStructure &ls);
void build_snk(const Topology &t, const Decomposition &d, SNKColumns &snk);
// The global near-kernel G (Sec. 4, "NK"): one column per interior vertex in
// dof_vert order, +1 on the unknown edges ending at it and -1 on those
// starting at it, rows ascending; sub = -1.
void build_nk(const Topology &t, SNKColumns &nk);

// kept vertices of an edge set: interior endpoints minus the highest vertex of
// every component (through edges between interior vertices) with no edge to a
// Dirichlet vertex; edge list given as unknown ids
std::vector<int32_t> kept_vertices(const Topology &t, const int32_t *dofs, int64_t count);

}  // namespace geneo
