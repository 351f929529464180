// Integer topology: structured Kuhn mesh, boundary, unknown numbering, CSR
// pattern, gather lists, box decomposition with overlap, partition of unity,
// local structures and split near-kernel columns.
//
// Mesh and boundary: Sec. 4 (Cartesian mesh, lowest-order Nedelec edges),
// Sec. 1 eq. "positivemaxwell" (E x n = 0 eliminated).  Decomposition: Sec. 2
// (R_i, eq. "PoU", eq. "k0", eq. "AS") and Sec. 4 ("one layer of elements
// is added in each direction").  Split near-kernel: Sec. 2, definition
// "near-kernelCS".
#include "topology.hpp"

#include <algorithm>
#include <numeric>
#include <stdexcept>

namespace geneo {

const int kDir[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0},
                        {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};

namespace {

// Kuhn walk orders (lexicographic permutations of the three axes)
const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
const int kLocalEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

int dir_of_offset(int dx, int dy, int dz) {
  for (int d = 0; d < 7; ++d)
    if (kDir[d][0] == dx && kDir[d][1] == dy && kDir[d][2] == dz) return d;
  return -1;
}

struct UnionFind {
  std::vector<int32_t> p;
  explicit UnionFind(size_t n) : p(n) { std::iota(p.begin(), p.end(), 0); }
  int32_t find(int32_t x) {
    while (p[x] != x) {
      p[x] = p[p[x]];
      x = p[x];
    }
    return x;
  }
  void unite(int32_t a, int32_t b) {
    a = find(a);
    b = find(b);
    if (a != b) p[std::max(a, b)] = std::min(a, b);
  }
};

}  // namespace

void build_topology(int nx, int ny, int nz, const double h[3], const uint8_t *active,
                    Topology &t, const uint8_t *natural) {
  t = Topology();
  t.nx = nx;
  t.ny = ny;
  t.nz = nz;
  for (int a = 0; a < 3; ++a) t.h[a] = h[a];
  const int64_t sx = 1, sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
  t.nverts = sz * (nz + 1);
  t.ncells = (int64_t)nx * ny * nz;
  const int64_t stride[3] = {sx, sy, sz};
  t.cell_rank.assign(t.ncells, -1);
  for (int64_t c = 0; c < t.ncells; ++c)
    if (active[c]) {
      t.cell_rank[c] = (int32_t)t.cells.size();
      t.cells.push_back((int32_t)c);
    }
  const int64_t nt = 6 * (int64_t)t.cells.size();
  t.tets.resize(nt * 4);
  t.tet_cell.resize(nt);
  for (size_t r = 0; r < t.cells.size(); ++r) {
    const int64_t c = t.cells[r];
    const int64_t i = c % nx, j = (c / nx) % ny, k = c / ((int64_t)nx * ny);
    const int64_t v0 = i + sy * j + sz * k;
    for (int p = 0; p < 6; ++p) {
      const int64_t v1 = v0 + stride[kPerm[p][0]];
      const int64_t v2 = v1 + stride[kPerm[p][1]];
      const int64_t v3 = v2 + stride[kPerm[p][2]];
      int32_t *tv = &t.tets[(6 * r + p) * 4];
      tv[0] = (int32_t)v0;
      tv[1] = (int32_t)v1;
      tv[2] = (int32_t)v2;
      tv[3] = (int32_t)v3;
      t.tet_cell[6 * r + p] = (int32_t)c;
    }
  }
  // edges by slot (lower vertex, direction); lexicographic (tail, head) order
  // is vertex-major with directions sorted by head offset
  std::vector<uint8_t> present(t.nverts * 7, 0);
  auto vijk = [&](int64_t v, int64_t &i, int64_t &j, int64_t &k) {
    i = v % (nx + 1);
    j = (v / (nx + 1)) % (ny + 1);
    k = v / sz;
  };
  std::vector<int32_t> slot_dir(nt * 6);
  for (int64_t tt = 0; tt < nt; ++tt) {
    const int32_t *tv = &t.tets[tt * 4];
    for (int e = 0; e < 6; ++e) {
      int64_t ai, aj, ak, bi, bj, bk;
      vijk(tv[kLocalEdge[e][0]], ai, aj, ak);
      vijk(tv[kLocalEdge[e][1]], bi, bj, bk);
      const int d = dir_of_offset((int)(bi - ai), (int)(bj - aj), (int)(bk - ak));
      if (d < 0) throw std::runtime_error("internal: non-Kuhn edge");
      slot_dir[tt * 6 + e] = d;
      present[(int64_t)tv[kLocalEdge[e][0]] * 7 + d] = 1;
    }
  }
  int order[7] = {0, 1, 2, 3, 4, 5, 6};
  auto off = [&](int d) { return kDir[d][0] * sx + kDir[d][1] * sy + kDir[d][2] * sz; };
  std::sort(order, order + 7, [&](int a, int b) { return off(a) < off(b); });
  std::vector<int32_t> slot_edge(t.nverts * 7, -1);
  for (int64_t v = 0; v < t.nverts; ++v)
    for (int q = 0; q < 7; ++q) {
      const int d = order[q];
      if (present[v * 7 + d]) {
        slot_edge[v * 7 + d] = (int32_t)t.edge_dir.size();
        t.edges.push_back((int32_t)v);
        t.edges.push_back((int32_t)(v + off(d)));
        t.edge_dir.push_back(d);
      }
    }
  const int64_t ne = t.nedges();
  t.tet_edges.resize(nt * 6);
  t.first_cell.assign(ne, INT32_MAX);
  for (int64_t tt = 0; tt < nt; ++tt)
    for (int e = 0; e < 6; ++e) {
      const int32_t id = slot_edge[(int64_t)t.tets[tt * 4 + kLocalEdge[e][0]] * 7 + slot_dir[tt * 6 + e]];
      t.tet_edges[tt * 6 + e] = id;
      t.first_cell[id] = std::min(t.first_cell[id], t.tet_cell[tt]);
    }
  // boundary: a square cell face whose neighbour cell is absent; both of its
  // triangles are boundary faces (exactly one incident active tetrahedron).
  // Dirichlet unless the cell marks that face natural.
  t.dir_edge.assign(ne, 0);
  t.dir_vert.assign(t.nverts, 0);
  t.used_vert.assign(t.nverts, 0);
  for (int64_t q = 0; q < nt * 4; ++q) t.used_vert[t.tets[q]] = 1;
  auto is_active = [&](int64_t i, int64_t j, int64_t k) {
    if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) return false;
    return active[i + nx * (j + (int64_t)ny * k)] != 0;
  };
  auto mark_edge = [&](int64_t v, int dx, int dy, int dz) {
    const int d = dir_of_offset(dx, dy, dz);
    const int32_t id = slot_edge[v * 7 + d];
    if (id < 0) throw std::runtime_error("internal: missing boundary edge");
    t.dir_edge[id] = 1;
  };
  for (int32_t c : t.cells) {
    const int64_t ci = c % nx, cj = (c / nx) % ny, ck = c / ((int64_t)nx * ny);
    const int64_t v0 = ci + sy * cj + sz * ck;
    for (int a = 0; a < 3; ++a)
      for (int side = 0; side < 2; ++side) {
        int64_t nb[3] = {ci, cj, ck};
        nb[a] += side ? 1 : -1;
        if (is_active(nb[0], nb[1], nb[2])) continue;
        if (natural && ((natural[c] >> (2 * a + side)) & 1)) continue;  // Neumann face
        // square face at coordinate a = side, spanned by the other axes b < c
        const int b = (a + 1) % 3 < (a + 2) % 3 ? (a + 1) % 3 : (a + 2) % 3;
        const int cc = 3 - a - b;
        const int64_t base = v0 + side * stride[a];
        const int64_t vb = base + stride[b], vc = base + stride[cc];
        const int64_t vbc = base + stride[b] + stride[cc];
        t.dir_vert[base] = t.dir_vert[vb] = t.dir_vert[vc] = t.dir_vert[vbc] = 1;
        int ub[3] = {0, 0, 0}, uc[3] = {0, 0, 0}, ubc[3] = {0, 0, 0};
        ub[b] = 1;
        uc[cc] = 1;
        ubc[b] = 1;
        ubc[cc] = 1;
        mark_edge(base, ub[0], ub[1], ub[2]);
        mark_edge(base, uc[0], uc[1], uc[2]);
        mark_edge(vb, uc[0], uc[1], uc[2]);
        mark_edge(vc, ub[0], ub[1], ub[2]);
        mark_edge(base, ubc[0], ubc[1], ubc[2]);
      }
  }
  t.edge_dof.assign(ne, -1);
  for (int64_t e = 0; e < ne; ++e)
    if (!t.dir_edge[e]) {
      t.edge_dof[e] = (int32_t)t.dof_edge.size();
      t.dof_edge.push_back((int32_t)e);
    }
  t.vert_dof.assign(t.nverts, -1);
  for (int64_t v = 0; v < t.nverts; ++v)
    if (t.used_vert[v] && !t.dir_vert[v]) {
      t.vert_dof[v] = (int32_t)t.dof_vert.size();
      t.dof_vert.push_back((int32_t)v);
    }
  // CSR pattern of A: unknowns sharing a tetrahedron
  const int64_t n = t.ndofs();
  std::vector<int64_t> cnt(n + 1, 0);
  for (int64_t tt = 0; tt < nt; ++tt)
    for (int a = 0; a < 6; ++a) {
      const int32_t r = t.edge_dof[t.tet_edges[tt * 6 + a]];
      if (r < 0) continue;
      for (int b = 0; b < 6; ++b)
        if (t.edge_dof[t.tet_edges[tt * 6 + b]] >= 0) cnt[r + 1]++;
    }
  for (int64_t r = 0; r < n; ++r) cnt[r + 1] += cnt[r];
  std::vector<int32_t> tmp(cnt[n]);
  {
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t tt = 0; tt < nt; ++tt)
      for (int a = 0; a < 6; ++a) {
        const int32_t r = t.edge_dof[t.tet_edges[tt * 6 + a]];
        if (r < 0) continue;
        for (int b = 0; b < 6; ++b) {
          const int32_t c2 = t.edge_dof[t.tet_edges[tt * 6 + b]];
          if (c2 >= 0) tmp[fill[r]++] = c2;
        }
      }
  }
  t.rowptr.assign(n + 1, 0);
  for (int64_t r = 0; r < n; ++r) {
    auto b = tmp.begin() + cnt[r], e = tmp.begin() + cnt[r + 1];
    std::sort(b, e);
    auto u = std::unique(b, e);
    t.col.insert(t.col.end(), b, u);
    t.rowptr[r + 1] = (int32_t)t.col.size();
  }
  // assembly gather lists (tet order within each nonzero)
  std::vector<int64_t> ccount(t.nnz() + 1, 0);
  std::vector<int32_t> epos(nt * 36, -1);
  for (int64_t tt = 0; tt < nt; ++tt)
    for (int a = 0; a < 6; ++a) {
      const int32_t r = t.edge_dof[t.tet_edges[tt * 6 + a]];
      if (r < 0) continue;
      for (int b = 0; b < 6; ++b) {
        const int32_t c2 = t.edge_dof[t.tet_edges[tt * 6 + b]];
        if (c2 < 0) continue;
        const int32_t *rb = t.col.data() + t.rowptr[r], *re = t.col.data() + t.rowptr[r + 1];
        const int32_t pos = (int32_t)(std::lower_bound(rb, re, c2) - t.col.data());
        epos[tt * 36 + a * 6 + b] = pos;
        ccount[pos + 1]++;
      }
    }
  for (int64_t k = 0; k < t.nnz(); ++k) ccount[k + 1] += ccount[k];
  t.cptr = ccount;
  t.cidx.resize(ccount[t.nnz()]);
  {
    std::vector<int64_t> fill(ccount.begin(), ccount.end() - 1);
    for (int64_t q = 0; q < nt * 36; ++q)
      if (epos[q] >= 0) t.cidx[fill[epos[q]]++] = (int32_t)q;
  }
  // load gather lists
  t.rptr.assign(n + 1, 0);
  for (int64_t tt = 0; tt < nt; ++tt)
    for (int a = 0; a < 6; ++a) {
      const int32_t r = t.edge_dof[t.tet_edges[tt * 6 + a]];
      if (r >= 0) t.rptr[r + 1]++;
    }
  for (int64_t r = 0; r < n; ++r) t.rptr[r + 1] += t.rptr[r];
  t.ridx.resize(t.rptr[n]);
  {
    std::vector<int64_t> fill(t.rptr.begin(), t.rptr.end() - 1);
    for (int64_t tt = 0; tt < nt; ++tt)
      for (int a = 0; a < 6; ++a) {
        const int32_t r = t.edge_dof[t.tet_edges[tt * 6 + a]];
        if (r >= 0) t.ridx[fill[r]++] = (int32_t)(tt * 6 + a);
      }
  }
}

void build_decomposition(const Topology &t, int px, int py, int pz, int overlap,
                         Decomposition &d, const int32_t *cell_part) {
  d = Decomposition();
  d.overlap = overlap;
  const int nx = t.nx, ny = t.ny, nz = t.nz;
  int64_t nb = (int64_t)px * py * pz;
  if (cell_part) {
    nb = 0;
    for (int32_t c : t.cells) nb = std::max<int64_t>(nb, (int64_t)cell_part[c] + 1);
  }
  std::vector<int32_t> bid(t.ncells, -1);
  std::vector<int32_t> renum(nb, -1);
  for (int32_t c : t.cells) {
    const int64_t i = c % nx, j = (c / nx) % ny, k = c / ((int64_t)nx * ny);
    const int64_t b = cell_part ? (int64_t)cell_part[c]
                                : i * px / nx + px * (j * py / ny + (int64_t)py * (k * pz / nz));
    bid[c] = (int32_t)b;
    renum[b] = 1;
  }
  for (int64_t b = 0; b < nb; ++b)
    if (renum[b] >= 0) renum[b] = d.nsub++;
  d.box_of_cell.assign(t.ncells, -1);
  for (int32_t c : t.cells) d.box_of_cell[c] = renum[bid[c]];
  d.sub_cells.resize(d.nsub);
  for (int32_t c : t.cells) d.sub_cells[d.box_of_cell[c]].push_back(c);
  // overlap: L dilations by vertex neighbours, restricted to active cells,
  // on the bounding region of each subdomain
  d.cell_mult.assign(t.ncells, 0);
  std::vector<uint8_t> mask(t.ncells, 0), next;
  for (int s = 0; s < d.nsub; ++s) {
    std::vector<int32_t> &cs = d.sub_cells[s];
    int64_t lo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, hi[3] = {-1, -1, -1};
    for (int32_t c : cs) {
      const int64_t q[3] = {c % nx, (c / nx) % ny, c / ((int64_t)nx * ny)};
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], q[a]);
        hi[a] = std::max(hi[a], q[a]);
      }
      mask[c] = 1;
    }
    const int64_t dims[3] = {nx, ny, nz};
    for (int layer = 0; layer < overlap; ++layer) {
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::max<int64_t>(0, lo[a] - 1);
        hi[a] = std::min<int64_t>(dims[a] - 1, hi[a] + 1);
      }
      std::vector<int32_t> add;
      for (int64_t k = lo[2]; k <= hi[2]; ++k)
        for (int64_t j = lo[1]; j <= hi[1]; ++j)
          for (int64_t i = lo[0]; i <= hi[0]; ++i) {
            const int64_t c = i + nx * (j + (int64_t)ny * k);
            if (mask[c] || t.cell_rank[c] < 0) continue;
            bool touch = false;
            for (int dk = -1; dk <= 1 && !touch; ++dk)
              for (int dj = -1; dj <= 1 && !touch; ++dj)
                for (int di = -1; di <= 1 && !touch; ++di) {
                  const int64_t a = i + di, b = j + dj, cc = k + dk;
                  if (a < 0 || b < 0 || cc < 0 || a >= nx || b >= ny || cc >= nz) continue;
                  if (mask[a + nx * (b + (int64_t)ny * cc)]) touch = true;
                }
            if (touch) add.push_back((int32_t)c);
          }
      for (int32_t c : add) mask[c] = 1;
      cs.insert(cs.end(), add.begin(), add.end());
    }
    std::sort(cs.begin(), cs.end());
    for (int32_t c : cs) {
      mask[c] = 0;
      d.cell_mult[c]++;
    }
  }
  d.k1 = 0;
  for (int32_t m : d.cell_mult) d.k1 = std::max(d.k1, m);
  // N_i: unknowns on the tetrahedra of Omega_i
  const int64_t n = t.ndofs();
  std::vector<uint8_t> seen(n, 0);
  d.N_off.assign(d.nsub + 1, 0);
  std::vector<int32_t> list;
  for (int s = 0; s < d.nsub; ++s) {
    list.clear();
    for (int32_t c : d.sub_cells[s]) {
      const int64_t r = t.cell_rank[c];
      for (int64_t tt = 6 * r; tt < 6 * r + 6; ++tt)
        for (int e = 0; e < 6; ++e) {
          const int32_t dof = t.edge_dof[t.tet_edges[tt * 6 + e]];
          if (dof >= 0 && !seen[dof]) {
            seen[dof] = 1;
            list.push_back(dof);
          }
        }
    }
    std::sort(list.begin(), list.end());
    for (int32_t dof : list) seen[dof] = 0;
    d.N_idx.insert(d.N_idx.end(), list.begin(), list.end());
    d.N_off[s + 1] = (int64_t)d.N_idx.size();
  }
  // Boolean partition of unity: owner = box of the lowest active cell holding the edge
  d.owner.resize(n);
  for (int64_t e = 0; e < n; ++e) d.owner[e] = d.box_of_cell[t.first_cell[t.dof_edge[e]]];
  // k0 = max_i #{j : R_j A R_i^T != 0}
  std::vector<int64_t> sp(n + 1, 0);
  for (int s = 0; s < d.nsub; ++s)
    for (int64_t q = d.N_off[s]; q < d.N_off[s + 1]; ++q) sp[d.N_idx[q] + 1]++;
  for (int64_t e = 0; e < n; ++e) sp[e + 1] += sp[e];
  std::vector<int32_t> subs(sp[n]);
  {
    std::vector<int64_t> fill(sp.begin(), sp.end() - 1);
    for (int s = 0; s < d.nsub; ++s)
      for (int64_t q = d.N_off[s]; q < d.N_off[s + 1]; ++q) subs[fill[d.N_idx[q]]++] = s;
  }
  std::vector<uint8_t> coupled((size_t)d.nsub * d.nsub, 0);
  for (int64_t r = 0; r < n; ++r)
    for (int32_t k = t.rowptr[r]; k < t.rowptr[r + 1]; ++k) {
      const int32_t c2 = t.col[k];
      for (int64_t a = sp[r]; a < sp[r + 1]; ++a)
        for (int64_t b = sp[c2]; b < sp[c2 + 1]; ++b)
          coupled[(size_t)subs[a] * d.nsub + subs[b]] = 1;
    }
  d.k0 = 0;
  for (int s = 0; s < d.nsub; ++s) {
    int c = 0;
    for (int q = 0; q < d.nsub; ++q) c += coupled[(size_t)s * d.nsub + q];
    d.k0 = std::max(d.k0, c);
  }
}

std::vector<int32_t> kept_vertices(const Topology &t, const int32_t *dofs, int64_t count) {
  std::vector<int32_t> verts;
  verts.reserve(2 * count);
  for (int64_t q = 0; q < count; ++q) {
    const int32_t e = t.dof_edge[dofs[q]];
    for (int s = 0; s < 2; ++s) {
      const int32_t v = t.edges[2 * e + s];
      if (t.vert_dof[v] >= 0) verts.push_back(v);
    }
  }
  std::sort(verts.begin(), verts.end());
  verts.erase(std::unique(verts.begin(), verts.end()), verts.end());
  auto idx = [&](int32_t v) {
    return (int32_t)(std::lower_bound(verts.begin(), verts.end(), v) - verts.begin());
  };
  UnionFind uf(verts.size());
  std::vector<uint8_t> anchored_v(verts.size(), 0);
  for (int64_t q = 0; q < count; ++q) {
    const int32_t e = t.dof_edge[dofs[q]];
    const int32_t a = t.edges[2 * e], b = t.edges[2 * e + 1];
    const bool ia = t.vert_dof[a] >= 0, ib = t.vert_dof[b] >= 0;
    if (ia && ib) uf.unite(idx(a), idx(b));
    else if (ia) anchored_v[idx(a)] = 1;
    else if (ib) anchored_v[idx(b)] = 1;
  }
  std::vector<uint8_t> anchored(verts.size(), 0);
  for (size_t k = 0; k < verts.size(); ++k)
    if (anchored_v[k]) anchored[uf.find((int32_t)k)] = 1;
  std::vector<int32_t> top(verts.size(), -1);
  for (size_t k = 0; k < verts.size(); ++k) {
    const int32_t r = uf.find((int32_t)k);
    if (!anchored[r]) top[r] = std::max(top[r], (int32_t)k);
  }
  std::vector<uint8_t> drop(verts.size(), 0);
  for (size_t k = 0; k < verts.size(); ++k)
    if (top[k] >= 0) drop[top[k]] = 1;
  std::vector<int32_t> out;
  for (size_t k = 0; k < verts.size(); ++k)
    if (!drop[k]) out.push_back(verts[k]);
  return out;
}

void build_local_structure(const Topology &t, const Decomposition &d, LocalStructure &ls) {
  ls = LocalStructure();
  const int64_t n = t.ndofs();
  const int64_t tot = d.N_off[d.nsub];
  std::vector<int32_t> g2l(n, -1);
  ls.lrowptr.assign(tot + 1, 0);
  ls.ncptr.assign(1, 0);
  ls.xv_off.assign(d.nsub + 1, 0);
  ls.gi_head.assign(tot, -1);
  ls.gi_tail.assign(tot, -1);
  ls.star_ptr.assign(1, 0);
  std::vector<int64_t> cnt;
  std::vector<int32_t> epos;
  for (int s = 0; s < d.nsub; ++s) {
    const int64_t o = d.N_off[s], ni = d.ni(s);
    for (int64_t r = 0; r < ni; ++r) g2l[d.N_idx[o + r]] = (int32_t)r;
    const int64_t lbase = (int64_t)ls.lcol.size();
    for (int64_t r = 0; r < ni; ++r) {
      const int32_t e = d.N_idx[o + r];
      for (int32_t k = t.rowptr[e]; k < t.rowptr[e + 1]; ++k) {
        const int32_t lc = g2l[t.col[k]];
        if (lc >= 0) {
          ls.lcol.push_back(lc);
          ls.lpos.push_back(k);
        }
      }
      ls.lrowptr[o + r + 1] = (int64_t)ls.lcol.size();
    }
    const int64_t lnnz = (int64_t)ls.lcol.size() - lbase;
    // A^Neu gather lists from the tetrahedra of Omega_s, tet order
    cnt.assign(lnnz + 1, 0);
    epos.clear();
    for (int32_t c : d.sub_cells[s]) {
      const int64_t rk = t.cell_rank[c];
      for (int64_t tt = 6 * rk; tt < 6 * rk + 6; ++tt)
        for (int a = 0; a < 6; ++a) {
          const int32_t ga = t.edge_dof[t.tet_edges[tt * 6 + a]];
          if (ga < 0) continue;
          const int32_t la = g2l[ga];
          for (int b = 0; b < 6; ++b) {
            const int32_t gb = t.edge_dof[t.tet_edges[tt * 6 + b]];
            if (gb < 0) continue;
            const int32_t lb = g2l[gb];
            const int32_t *cb = ls.lcol.data() + ls.lrowptr[o + la];
            const int32_t *ce = ls.lcol.data() + ls.lrowptr[o + la + 1];
            const int64_t p = (std::lower_bound(cb, ce, lb) - ls.lcol.data()) - lbase;
            epos.push_back((int32_t)p);
            epos.push_back((int32_t)(tt * 36 + a * 6 + b));
            cnt[p + 1]++;
          }
        }
    }
    for (int64_t k = 0; k < lnnz; ++k) cnt[k + 1] += cnt[k];
    const int64_t nbase = (int64_t)ls.ncidx.size();
    ls.ncidx.resize(nbase + cnt[lnnz]);
    {
      std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
      for (size_t q = 0; q < epos.size(); q += 2)
        ls.ncidx[nbase + fill[epos[q]]++] = epos[q + 1];
    }
    for (int64_t k = 0; k < lnnz; ++k) ls.ncptr.push_back(nbase + cnt[k + 1]);
    // kept vertices of N_s and the local gradient G_s
    std::vector<int32_t> kv = kept_vertices(t, d.N_idx.data() + o, ni);
    ls.xv_vert.insert(ls.xv_vert.end(), kv.begin(), kv.end());
    ls.xv_off[s + 1] = (int64_t)ls.xv_vert.size();
    auto vidx = [&](int32_t v) -> int32_t {
      auto it = std::lower_bound(kv.begin(), kv.end(), v);
      return (it != kv.end() && *it == v) ? (int32_t)(it - kv.begin()) : -1;
    };
    std::vector<std::vector<std::pair<int32_t, int8_t>>> star(kv.size());
    for (int64_t r = 0; r < ni; ++r) {
      const int32_t e = t.dof_edge[d.N_idx[o + r]];
      const int32_t hv = vidx(t.edges[2 * e + 1]), tv = vidx(t.edges[2 * e]);
      ls.gi_head[o + r] = hv;
      ls.gi_tail[o + r] = tv;
      if (hv >= 0) star[hv].push_back({(int32_t)r, (int8_t)1});
      if (tv >= 0) star[tv].push_back({(int32_t)r, (int8_t)-1});
    }
    for (auto &st : star) {
      for (auto &p : st) {
        ls.star_row.push_back(p.first);
        ls.star_sgn.push_back(p.second);
      }
      ls.star_ptr.push_back((int64_t)ls.star_row.size());
    }
    for (int64_t r = 0; r < ni; ++r) g2l[d.N_idx[o + r]] = -1;
  }
  // prolongation map
  ls.g2l_ptr.assign(n + 1, 0);
  for (int64_t q = 0; q < tot; ++q) ls.g2l_ptr[d.N_idx[q] + 1]++;
  for (int64_t e = 0; e < n; ++e) ls.g2l_ptr[e + 1] += ls.g2l_ptr[e];
  ls.g2l_slot.resize(tot);
  std::vector<int64_t> fill(ls.g2l_ptr.begin(), ls.g2l_ptr.end() - 1);
  for (int64_t q = 0; q < tot; ++q) ls.g2l_slot[fill[d.N_idx[q]]++] = q;
}

void build_nk(const Topology &t, SNKColumns &nk) {
  nk = SNKColumns();
  const int64_t nv = (int64_t)t.dof_vert.size();
  const int64_t n = t.ndofs();
  // A connected component of unknown edges with no edge to a Dirichlet
  // vertex (every boundary face natural) carries the constant in the kernel
  // of G: its highest vertex is dropped so that Z = G keeps full column rank
  // and E = G^T A G stays SPD (Sec. 3.2 needs a full-rank Z).
  std::vector<int32_t> all(n);
  for (int64_t r = 0; r < n; ++r) all[r] = (int32_t)r;
  const std::vector<int32_t> kv = kept_vertices(t, all.data(), n);
  std::vector<int32_t> col_of(nv, -1);  // vertex unknown -> column
  for (size_t q = 0; q < kv.size(); ++q) col_of[t.vert_dof[kv[q]]] = (int32_t)q;
  const int64_t ncol = (int64_t)kv.size();
  std::vector<int64_t> cnt(ncol + 1, 0);
  for (int64_t r = 0; r < n; ++r) {
    const int32_t e = t.dof_edge[r];
    for (int s = 0; s < 2; ++s) {
      const int32_t k = t.vert_dof[t.edges[2 * e + s]];
      if (k >= 0 && col_of[k] >= 0) cnt[col_of[k] + 1]++;
    }
  }
  for (int64_t k = 0; k < ncol; ++k) cnt[k + 1] += cnt[k];
  nk.ptr = cnt;
  nk.row.assign(cnt[ncol], 0);
  nk.sgn.assign(cnt[ncol], 0);
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  for (int64_t r = 0; r < n; ++r) {  // rows visited in ascending order
    const int32_t e = t.dof_edge[r];
    for (int s = 0; s < 2; ++s) {
      const int32_t k = t.vert_dof[t.edges[2 * e + s]];
      if (k < 0 || col_of[k] < 0) continue;
      const int32_t q = col_of[k];
      nk.row[fill[q]] = (int32_t)r;
      nk.sgn[fill[q]] = s ? 1 : -1;  // head +1, tail -1
      ++fill[q];
    }
  }
  nk.sub.assign(ncol, -1);
  nk.vert.assign(kv.begin(), kv.end());
}

void build_snk(const Topology &t, const Decomposition &d, SNKColumns &snk) {
  snk = SNKColumns();
  snk.ptr.push_back(0);
  std::vector<int32_t> owned;
  for (int s = 0; s < d.nsub; ++s) {
    owned.clear();
    for (int64_t q = d.N_off[s]; q < d.N_off[s + 1]; ++q)
      if (d.owner[d.N_idx[q]] == s) owned.push_back(d.N_idx[q]);
    std::vector<int32_t> kv = kept_vertices(t, owned.data(), (int64_t)owned.size());
    std::vector<std::vector<std::pair<int32_t, int8_t>>> col(kv.size());
    for (int32_t dof : owned) {
      const int32_t e = t.dof_edge[dof];
      for (int sd = 0; sd < 2; ++sd) {
        const int32_t v = t.edges[2 * e + sd];
        auto it = std::lower_bound(kv.begin(), kv.end(), v);
        if (it != kv.end() && *it == v) col[it - kv.begin()].push_back({dof, (int8_t)(sd ? 1 : -1)});
      }
    }
    for (size_t k = 0; k < kv.size(); ++k) {
      std::sort(col[k].begin(), col[k].end());
      snk.sub.push_back(s);
      snk.vert.push_back(kv[k]);
      for (auto &p : col[k]) {
        snk.row.push_back(p.first);
        snk.sgn.push_back(p.second);
      }
      snk.ptr.push_back((int64_t)snk.row.size());
    }
  }
}

}  // namespace geneo
