// Numerical set-up on the GPU: Whitney element matrices, assembly of A, the
// local Dirichlet matrices and their explicit inverses, the split
// near-kernel coarse basis Z and the coarse matrix E = Z^T A Z with its
// inverse.
//
// Element matrices: Sec. 2, eq. "bilinearformposmax" with lowest-order
// Nedelec (Whitney) functions W_ab = l_a grad l_b - l_b grad l_a,
// curl W_ab = 2 grad l_a x grad l_b, int l_i l_j = |T| (1 + d_ij) / 20.
// A = K + gamma M: Sec. 1, eq. "discretemaxwell".  A_i = R_i A R_i^T:
// Sec. 2, eq. "AS".  Z and E: Sec. 2 (definition "near-kernelCS",
// E = Z^T A Z).
#include <algorithm>
#include <chrono>
#include <functional>

#include "ctx.hpp"
#include "ordered_drop.hpp"
#include "setup.hpp"
#include "xi.hpp"

namespace geneo {

// ---------------------------------------------------------------------------
// element matrices

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// barycentric gradients and volume of a tetrahedron of the structured mesh
__device__ void tet_geometry(const int32_t *tv, int nx, int ny, double hx, double hy, double hz,
                             double g[4][3], double &vol) {
  double p[4][3];
  for (int q = 0; q < 4; ++q) {
    const int64_t v = tv[q];
    const int64_t i = v % (nx + 1), j = (v / (nx + 1)) % (ny + 1),
                  k = v / ((int64_t)(nx + 1) * (ny + 1));
    p[q][0] = i * hx;
    p[q][1] = j * hy;
    p[q][2] = k * hz;
  }
  double r1[3], r2[3], r3[3];
  for (int d = 0; d < 3; ++d) {
    r1[d] = p[1][d] - p[0][d];
    r2[d] = p[2][d] - p[0][d];
    r3[d] = p[3][d] - p[0][d];
  }
  double c23[3], c31[3], c12[3];
  cross3(r2, r3, c23);
  cross3(r3, r1, c31);
  cross3(r1, r2, c12);
  const double det = r1[0] * c23[0] + r1[1] * c23[1] + r1[2] * c23[2];
  for (int d = 0; d < 3; ++d) {
    g[1][d] = c23[d] / det;
    g[2][d] = c31[d] / det;
    g[3][d] = c12[d] / det;
    g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
  }
  vol = fabs(det) / 6.0;
}

__constant__ int c_le[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

// curl-curl and mass element matrices (upper triangle computed, mirrored)
__device__ void element_KM(const double g[4][3], double vol, double K[6][6], double M[6][6]) {
  double curl[6][3];
  for (int e = 0; e < 6; ++e) {
    cross3(g[c_le[e][0]], g[c_le[e][1]], curl[e]);
    for (int d = 0; d < 3; ++d) curl[e][d] *= 2.0;
  }
  double G[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) G[a][b] = g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2];
  const double w = vol / 20.0;
  for (int e = 0; e < 6; ++e)
    for (int f = e; f < 6; ++f) {
      const int a = c_le[e][0], b = c_le[e][1], c = c_le[f][0], d = c_le[f][1];
      const double kk = vol * (curl[e][0] * curl[f][0] + curl[e][1] * curl[f][1] + curl[e][2] * curl[f][2]);
      const double mm = w * ((1.0 + (a == c)) * G[b][d] - (1.0 + (a == d)) * G[b][c] -
                             (1.0 + (b == c)) * G[a][d] + (1.0 + (b == d)) * G[a][c]);
      K[e][f] = K[f][e] = kk;
      M[e][f] = M[f][e] = mm;
    }
}

__global__ void k_element(const int32_t *__restrict__ tets, const int32_t *__restrict__ tet_cell,
                          const double *__restrict__ mu, const double *__restrict__ eps,
                          double gamma, int nx, int ny, double hx, double hy, double hz,
                          int64_t ntets, double *__restrict__ Ae) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ntets) return;
  double g[4][3], vol, K[6][6], M[6][6];
  tet_geometry(tets + 4 * t, nx, ny, hx, hy, hz, g, vol);
  element_KM(g, vol, K, M);
  const int c = tet_cell[t];
  const double mi = mu[c], ep = eps[c] * gamma;
  for (int e = 0; e < 6; ++e)
    for (int f = 0; f < 6; ++f) Ae[t * 36 + e * 6 + f] = mi * K[e][f] + ep * M[e][f];
}

// per tetrahedron: mc[t][a] = sum_b M1_T[a][b] c[edge_b] (eps = 1 mass)
__global__ void k_rhs_element(const int32_t *__restrict__ tets, const int32_t *__restrict__ tet_edges,
                              const double *__restrict__ cedge, int nx, int ny, double hx,
                              double hy, double hz, int64_t ntets, double *__restrict__ mc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ntets) return;
  double g[4][3], vol, K[6][6], M[6][6];
  tet_geometry(tets + 4 * t, nx, ny, hx, hy, hz, g, vol);
  element_KM(g, vol, K, M);
  double cv[6];
  for (int b = 0; b < 6; ++b) cv[b] = cedge[tet_edges[6 * t + b]];
  for (int a = 0; a < 6; ++a) {
    double s = 0;
    for (int b = 0; b < 6; ++b) s = fma(M[a][b], cv[b], s);
    mc[6 * t + a] = s;
  }
}

// c_e = f(slot of e) . (x_head - x_tail)
__global__ void k_rhs_edge(const double *__restrict__ fslot, const int32_t *__restrict__ tail,
                           const int32_t *__restrict__ dir, double hx, double hy, double hz,
                           int64_t nedges, double *__restrict__ cedge) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nedges) return;
  const int d = dir[e];
  const int dx[7] = {1, 0, 0, 1, 1, 0, 1}, dy[7] = {0, 1, 0, 1, 0, 1, 1}, dz[7] = {0, 0, 1, 0, 1, 1, 1};
  const double *f = fslot + ((int64_t)tail[e] * 7 + d) * 3;
  cedge[e] = f[0] * (dx[d] * hx) + f[1] * (dy[d] * hy) + f[2] * (dz[d] * hz);
}

// b_e = sum over its (tet, local edge) slots, in tet order
__global__ void k_gather_sum(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                             const double *__restrict__ src, int64_t n, double *__restrict__ out) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  double s = 0;
  for (int64_t k = ptr[r]; k < ptr[r + 1]; ++k) s += src[idx[k]];
  out[r] = s;
}

// A_i -> tile-packed lower storage (diagonal tiles full)
__global__ void k_extract_local(const int64_t *__restrict__ Noff, const int64_t *__restrict__ lrowptr,
                                const int32_t *__restrict__ lcol, const int32_t *__restrict__ lpos,
                                const double *__restrict__ val, const int64_t *__restrict__ toff,
                                double *__restrict__ tiles) {
  const int m = blockIdx.y;
  const int64_t ni = Noff[m + 1] - Noff[m];
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < ni;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t slot = Noff[m] + r;
    const int I = (int)(r / kTile), rr = (int)(r % kTile);
    for (int64_t k = lrowptr[slot]; k < lrowptr[slot + 1]; ++k) {
      const int c = lcol[k];
      const int J = c / kTile;
      if (J > I) continue;
      tiles[(toff[m] + (int64_t)I * (I + 1) / 2 + J) * kTileElems + rr * kTile + (c % kTile)] = val[lpos[k]];
    }
  }
}

__device__ __forceinline__ double csr_lookup(const int32_t *rowptr, const int32_t *col,
                                             const double *val, int32_t r, int32_t c) {
  int lo = rowptr[r], hi = rowptr[r + 1] - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int32_t v = col[mid];
    if (v == c) return val[mid];
    if (v < c) lo = mid + 1;
    else hi = mid - 1;
  }
  return 0.0;
}

// Column-tetrahedron incidence of the coarse basis.  For column a and a
// tetrahedron T touching its support, entry q stores 15 doubles:
//   [0..2]  sqrt(mu^-1_T |T|) * sum_e z_e curl W_e   (curl of the column on T)
//   [3..8]  z_e on the six local edges (0 off the support)
//   [9..14] gamma eps_T M_T z
// so that E[a][b] = sum over common T of c_a . c_b + z_a . m_b, which equals
// Z^T A Z while the K-part of gradient columns never cancels in assembled A.
__global__ void k_coltet(const int32_t *__restrict__ ct_tet, int64_t nent,
                         const int32_t *__restrict__ tets, const int32_t *__restrict__ tet_cell,
                         const double *__restrict__ mu, const double *__restrict__ eps,
                         double gamma, int nx, int ny, double hx, double hy, double hz,
                         double *__restrict__ ct) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nent) return;
  const int32_t t = ct_tet[q];
  double g[4][3], vol, K[6][6], M[6][6];
  tet_geometry(tets + 4 * (int64_t)t, nx, ny, hx, hy, hz, g, vol);
  element_KM(g, vol, K, M);
  double *e = ct + q * 15;
  double z[6];
  for (int k = 0; k < 6; ++k) z[k] = e[3 + k];
  const int cell = tet_cell[t];
  const double sc = sqrt(mu[cell] * vol), ge = gamma * eps[cell];
  double c[3] = {0, 0, 0};
  for (int k = 0; k < 6; ++k) {
    if (z[k] == 0.0) continue;
    double cw[3];
    cross3(g[c_le[k][0]], g[c_le[k][1]], cw);
    for (int d = 0; d < 3; ++d) c[d] = fma(2.0 * z[k], cw[d], c[d]);
  }
  for (int d = 0; d < 3; ++d) e[d] = sc * c[d];
  for (int a = 0; a < 6; ++a) {
    double v = 0;
    for (int b = 0; b < 6; ++b) v = fma(M[a][b], z[b], v);
    e[9 + a] = ge * v;
  }
}

// (X^T A X)[a][b] for the lower pattern of each matrix of a tile batch:
// column a belongs to matrix cmat[a] at local index cloc[a]; iterates over
// the shorter tet list and binary-searches the longer one.
__global__ void k_galerkin(const int64_t *__restrict__ pptr, const int32_t *__restrict__ pcol,
                           int64_t ncols, const int64_t *__restrict__ ct_ptr,
                           const int32_t *__restrict__ ct_tet, const double *__restrict__ ct,
                           const int32_t *__restrict__ cmat, const int32_t *__restrict__ cloc,
                           const int64_t *__restrict__ toff, double *__restrict__ tiles) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.y + threadIdx.y;
  if (a >= ncols) return;
  for (int64_t q = pptr[a] + threadIdx.x; q < pptr[a + 1]; q += blockDim.x) {
    const int64_t b = pcol[q];
    const int64_t sa = ct_ptr[a], ea = ct_ptr[a + 1], sb = ct_ptr[b], eb = ct_ptr[b + 1];
    const bool swap = (ea - sa) > (eb - sb);
    const int64_t xs = swap ? sb : sa, xe = swap ? eb : ea, ys = swap ? sa : sb, ye = swap ? ea : eb;
    double s = 0;
    for (int64_t i = xs; i < xe; ++i) {
      const int32_t t = ct_tet[i];
      int64_t lo = ys, hi = ye - 1, hit = -1;
      while (lo <= hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int32_t v = ct_tet[mid];
        if (v == t) {
          hit = mid;
          break;
        }
        if (v < t) lo = mid + 1;
        else hi = mid - 1;
      }
      if (hit < 0) continue;
      const double *ea_ = ct + (swap ? hit : i) * 15;  // entry of column a
      const double *eb_ = ct + (swap ? i : hit) * 15;  // entry of column b
      double v = ea_[0] * eb_[0] + ea_[1] * eb_[1] + ea_[2] * eb_[2];
      for (int k = 0; k < 6; ++k) v = fma(ea_[3 + k], eb_[9 + k], v);
      s += v;
    }
    const int m = cmat[a];
    const int64_t la = cloc[a], lb = cloc[b];
    const int I = (int)(la / kTile), J = (int)(lb / kTile);
    const int64_t tb = (toff[m] + (int64_t)I * (I + 1) / 2 + J) * kTileElems;
    tiles[tb + (la % kTile) * kTile + (lb % kTile)] = s;
    if (I == J) tiles[tb + (lb % kTile) * kTile + (la % kTile)] = s;
  }
}

__global__ void k_set_diag(double *tiles, const int64_t *toff, int m, int64_t r0, int64_t r1) {
  const int64_t r = r0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= r1) return;
  const int I = (int)(r / kTile);
  tiles[(toff[m] + (int64_t)I * (I + 1) / 2 + I) * kTileElems + (r % kTile) * (kTile + 1)] = 1.0;
}

__global__ void k_take(const double *__restrict__ src, const int32_t *__restrict__ idx,
                       double *__restrict__ dst, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

// per tetrahedron: scaled curls (18) and gamma eps M_T (36)
__global__ void k_tet_ops(const int32_t *__restrict__ tets, const int32_t *__restrict__ tet_cell,
                          const double *__restrict__ mu, const double *__restrict__ eps,
                          double gamma, int nx, int ny, double hx, double hy, double hz,
                          int64_t ntets, double *__restrict__ tcurl, double *__restrict__ tmass) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ntets) return;
  double g[4][3], vol, K[6][6], M[6][6];
  tet_geometry(tets + 4 * t, nx, ny, hx, hy, hz, g, vol);
  element_KM(g, vol, K, M);
  const int cell = tet_cell[t];
  const double sc = sqrt(mu[cell] * vol), ge = gamma * eps[cell];
  for (int e = 0; e < 6; ++e) {
    double cw[3];
    cross3(g[c_le[e][0]], g[c_le[e][1]], cw);
    for (int d = 0; d < 3; ++d) tcurl[t * 18 + e * 3 + d] = sc * 2.0 * cw[d];
    for (int f = 0; f < 6; ++f) tmass[t * 36 + e * 6 + f] = ge * M[e][f];
  }
}

void tet_operators(geneo_ctx *c, DevBuf<double> &tcurl, DevBuf<double> &tmass, cudaStream_t s) {
  const int64_t nt = c->topo.ntets();
  tcurl.alloc(nt * 18);
  tmass.alloc(nt * 36);
  k_tet_ops<<<grid_for(nt, 128), 128, 0, s>>>(c->d_tets.p, c->d_tet_cell.p, c->d_mu.p, c->d_eps.p,
                                              c->gamma, c->nx, c->ny, c->h[0], c->h[1], c->h[2], nt,
                                              tcurl.p, tmass.p);
  GENEO_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------

void check_device_error(geneo_ctx *c, cudaStream_t s) {
  GENEO_CUDA(cudaStreamSynchronize(s));
  int e = 0;
  GENEO_CUDA(cudaMemcpy(&e, c->d_err.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (e == kDevNotSPD) throw Error(GENEO_ERR_NOT_SPD, "a factorisation pivot was not positive");
  if (e == kDevTimeout) throw Error(GENEO_ERR_TIMEOUT, "a bounded device wait gave up");
  if (e != 0) throw Error(GENEO_ERR_CUDA, "device error word set");
}

static void build_z_csr(geneo_ctx *c) {
  const int64_t n = c->topo.ndofs();
  std::vector<int64_t> rp(n + 1, 0);
  for (int32_t r : c->zc_row) rp[r + 1]++;
  for (int64_t e = 0; e < n; ++e) rp[e + 1] += rp[e];
  std::vector<int32_t> rc(c->zc_row.size());
  std::vector<double> rv(c->zc_row.size());
  std::vector<int64_t> fill(rp.begin(), rp.end() - 1);
  for (int64_t a = 0; a < c->n0; ++a)
    for (int64_t k = c->zc_ptr[a]; k < c->zc_ptr[a + 1]; ++k) {
      const int32_t r = c->zc_row[k];
      rc[fill[r]] = (int32_t)a;
      rv[fill[r]++] = c->zc_val[k];
    }
  c->d_zc_ptr.upload(c->zc_ptr, c->stream);
  c->d_zc_row.upload(c->zc_row, c->stream);
  c->d_zc_val.upload(c->zc_val, c->stream);
  c->d_zr_ptr.upload(rp, c->stream);
  c->d_zr_col.upload(rc, c->stream);
  c->d_zr_val.upload(rv, c->stream);
  GENEO_CUDA(cudaStreamSynchronize(c->stream));
}

// Column-tetrahedron lists of sparse columns: for each column the sorted
// tetrahedra touching its support (only those of Omega_mat when X.neumann),
// with the 15-double entries of k_coltet computed on the device.
void coltet_build(geneo_ctx *c, const Columns &X, std::vector<int64_t> &ct_ptr,
                  std::vector<int32_t> &ct_tet, DevBuf<int64_t> &dctp, DevBuf<int32_t> &dctt,
                  DevBuf<double> &dct, cudaStream_t s) {
  const Topology &t = c->topo;
  const int64_t n = t.ndofs(), nt = t.ntets(), ncol = (int64_t)X.mat.size();
  // unknown -> tetrahedra
  std::vector<int64_t> tp(n + 1, 0);
  for (int64_t q = 0; q < nt * 6; ++q) {
    const int32_t d = t.edge_dof[t.tet_edges[q]];
    if (d >= 0) tp[d + 1]++;
  }
  for (int64_t e = 0; e < n; ++e) tp[e + 1] += tp[e];
  std::vector<int32_t> tl(tp[n]);
  {
    std::vector<int64_t> fill(tp.begin(), tp.end() - 1);
    for (int64_t q = 0; q < nt * 6; ++q) {
      const int32_t d = t.edge_dof[t.tet_edges[q]];
      if (d >= 0) tl[fill[d]++] = (int32_t)(q / 6);
    }
  }
  ct_ptr.assign(1, 0);
  ct_tet.clear();
  std::vector<double> ct;
  std::vector<double> val(n, 0.0);
  std::vector<uint8_t> in(n, 0);
  std::vector<int32_t> tets;
  for (int64_t a = 0; a < ncol; ++a) {
    tets.clear();
    for (int64_t k = X.ptr[a]; k < X.ptr[a + 1]; ++k) {
      const int32_t e = X.row[k];
      val[e] = X.val[k];
      in[e] = 1;
      tets.insert(tets.end(), tl.begin() + tp[e], tl.begin() + tp[e + 1]);
    }
    std::sort(tets.begin(), tets.end());
    tets.erase(std::unique(tets.begin(), tets.end()), tets.end());
    const std::vector<int32_t> *cells = X.neumann ? &c->dec.sub_cells[X.mat[a]] : nullptr;
    for (int32_t tt : tets) {
      if (cells && !std::binary_search(cells->begin(), cells->end(), t.tet_cell[tt])) continue;
      ct_tet.push_back(tt);
      double ent[15] = {0};
      for (int k = 0; k < 6; ++k) {
        const int32_t d = t.edge_dof[t.tet_edges[(int64_t)tt * 6 + k]];
        if (d >= 0 && in[d]) ent[3 + k] = val[d];
      }
      ct.insert(ct.end(), ent, ent + 15);
    }
    ct_ptr.push_back((int64_t)ct_tet.size());
    for (int64_t k = X.ptr[a]; k < X.ptr[a + 1]; ++k) {
      val[X.row[k]] = 0.0;
      in[X.row[k]] = 0;
    }
  }
  dctp.upload(ct_ptr, s);
  dctt.upload(ct_tet, s);
  dct.upload(ct, s);
  if (dctt.n)
    k_coltet<<<grid_for(dctt.n, 128), 128, 0, s>>>(dctt.p, dctt.n, c->d_tets.p, c->d_tet_cell.p,
                                                   c->d_mu.p, c->d_eps.p, c->gamma, c->nx, c->ny,
                                                   c->h[0], c->h[1], c->h[2], dct.p);
  GENEO_CHECK_LAUNCH();
  GENEO_CUDA(cudaStreamSynchronize(s));
}

// Galerkin plan of sparse columns: column-tetrahedron entries on the device
// and the lower pattern (pairs of columns of the same matrix sharing a
// tetrahedron, b with loc(b) <= loc(a), per column a, ascending b).
void galerkin_plan(geneo_ctx *c, const Columns &X, GalerkinPlan &P, cudaStream_t s) {
  const Topology &t = c->topo;
  const int64_t nt = t.ntets(), ncol = (int64_t)X.mat.size();
  P.ncol = ncol;
  std::vector<int64_t> ct_ptr;
  std::vector<int32_t> ct_tet;
  coltet_build(c, X, ct_ptr, ct_tet, P.dctp, P.dctt, P.dct, s);
  std::vector<int64_t> tcp(nt + 1, 0);
  for (int32_t tt : ct_tet) tcp[tt + 1]++;
  for (int64_t q = 0; q < nt; ++q) tcp[q + 1] += tcp[q];
  std::vector<int32_t> tcl(ct_tet.size());
  {
    std::vector<int64_t> fill(tcp.begin(), tcp.end() - 1);
    for (int64_t a = 0; a < ncol; ++a)
      for (int64_t q = ct_ptr[a]; q < ct_ptr[a + 1]; ++q) tcl[fill[ct_tet[q]]++] = (int32_t)a;
  }
  P.pptr.assign(1, 0);
  P.pcol.clear();
  std::vector<int32_t> list;
  std::vector<uint8_t> mark(ncol, 0);
  for (int64_t a = 0; a < ncol; ++a) {
    list.clear();
    for (int64_t q = ct_ptr[a]; q < ct_ptr[a + 1]; ++q) {
      const int32_t tt = ct_tet[q];
      for (int64_t u = tcp[tt]; u < tcp[tt + 1]; ++u) {
        const int32_t bb = tcl[u];
        if (X.mat[bb] == X.mat[a] && X.loc[bb] <= X.loc[a] && !mark[bb]) {
          mark[bb] = 1;
          list.push_back(bb);
        }
      }
    }
    std::sort(list.begin(), list.end());
    for (int32_t bb : list) mark[bb] = 0;
    P.pcol.insert(P.pcol.end(), list.begin(), list.end());
    P.pptr.push_back((int64_t)P.pcol.size());
  }
  P.dpp.upload(P.pptr, s);
  P.dpc.upload(P.pcol, s);
  GENEO_CUDA(cudaStreamSynchronize(s));
}

// vals[q] = (X^T A X)[a][pcol[q]] for every pattern entry q
__global__ void k_galerkin_vals(const int64_t *__restrict__ pptr, const int32_t *__restrict__ pcol,
                                int64_t ncols, const int64_t *__restrict__ ct_ptr,
                                const int32_t *__restrict__ ct_tet, const double *__restrict__ ct,
                                double *__restrict__ vals) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.y + threadIdx.y;
  if (a >= ncols) return;
  for (int64_t q = pptr[a] + threadIdx.x; q < pptr[a + 1]; q += blockDim.x) {
    const int64_t b = pcol[q];
    const int64_t sa = ct_ptr[a], ea = ct_ptr[a + 1], sb = ct_ptr[b], eb = ct_ptr[b + 1];
    const bool swap = (ea - sa) > (eb - sb);
    const int64_t xs = swap ? sb : sa, xe = swap ? eb : ea, ys = swap ? sa : sb, ye = swap ? ea : eb;
    double s = 0;
    for (int64_t i = xs; i < xe; ++i) {
      const int32_t t = ct_tet[i];
      int64_t lo = ys, hi = ye - 1, hit = -1;
      while (lo <= hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int32_t v = ct_tet[mid];
        if (v == t) {
          hit = mid;
          break;
        }
        if (v < t) lo = mid + 1;
        else hi = mid - 1;
      }
      if (hit < 0) continue;
      const double *ea_ = ct + (swap ? hit : i) * 15;
      const double *eb_ = ct + (swap ? i : hit) * 15;
      double v = ea_[0] * eb_[0] + ea_[1] * eb_[1] + ea_[2] * eb_[2];
      for (int k = 0; k < 6; ++k) v = fma(ea_[3 + k], eb_[9 + k], v);
      s += v;
    }
    vals[q] = s;
  }
}

void galerkin_values(GalerkinPlan &P, double *vals, cudaStream_t s) {
  if (P.ncol == 0) return;
  k_galerkin_vals<<<grid_for(P.ncol, 8), dim3(32, 8), 0, s>>>(P.dpp.p, P.dpc.p, P.ncol, P.dctp.p,
                                                             P.dctt.p, P.dct.p, vals);
  GENEO_CHECK_LAUNCH();
}

// X^T A X for the columns, element by element through per-tet curls (see
// k_coltet), written into `tiles` of batch b at (cloc[a], cloc[b]).
void galerkin_tiles(geneo_ctx *c, const Columns &X, TileBatch &b, double *tiles, cudaStream_t s) {
  const int64_t ncol = (int64_t)X.mat.size();
  if (ncol == 0) return;
  GalerkinPlan P;
  galerkin_plan(c, X, P, s);
  DevBuf<int32_t> dmat, dloc;
  dmat.upload(X.mat, s);
  dloc.upload(X.loc, s);
  k_galerkin<<<grid_for(ncol, 8), dim3(32, 8), 0, s>>>(P.dpp.p, P.dpc.p, ncol, P.dctp.p,
                                                      P.dctt.p, P.dct.p, dmat.p, dloc.p,
                                                      b.d_toff.p, tiles);
  GENEO_CHECK_LAUNCH();
  GENEO_CUDA(cudaStreamSynchronize(s));
}

// Coarse columns as Galerkin input; column a placed at local index loc(a)
static Columns coarse_columns(const geneo_ctx *c, int64_t gap_after_snk) {
  Columns X;
  for (int64_t a = 0; a < c->n0; ++a) {
    for (int64_t k = c->zc_ptr[a]; k < c->zc_ptr[a + 1]; ++k) {
      X.row.push_back(c->zc_row[k]);
      X.val.push_back(c->zc_val[k]);
    }
    X.ptr.push_back((int64_t)X.row.size());
    X.mat.push_back(0);
    X.loc.push_back((int32_t)(a < c->n0_snk ? a : a + gap_after_snk));
  }
  return X;
}

// Z must be a full-rank basis of V_G + V_GenEO (Sec. 3.2, eq. "V0GenEOAS"):
// drop GenEO columns whose pivot in the ordered Cholesky of the GenEO Schur
// complement E_hh - E_hg E_gg^-1 E_gh is below kDepTol times their diagonal.
constexpr double kDepTol = 1e-8;

static void apply_geneo_keep(geneo_ctx *c, const std::vector<int64_t> &keep);

// The same filter through the multifrontal: the root front holds the GenEO
// columns, so after the fronts below it are factored its pivot block is the
// Schur complement, without a dense matrix over the split near-kernel.
static void geneo_filter_mf(geneo_ctx *c) {
  MfSchur sc;
  mf_setup(c, &sc);
  apply_geneo_keep(c, ordered_drop(sc.S, sc.diag, sc.nh, kDepTol));
}

static void geneo_filter(geneo_ctx *c) {
  cudaStream_t s = c->stream;
  const int64_t ns = c->n0_snk, nh = c->n0_geneo;
  const int64_t off = (ns + kTile - 1) / kTile * kTile;
  TileBatch fb;
  fb.layout({off + nh});
  fb.upload_meta(s);
  DevBuf<double> tiles;
  tiles.alloc(tile_elems(fb));
  tiles_init_padding(fb, tiles.p, s);
  if (off > ns) k_set_diag<<<1, 64, 0, s>>>(tiles.p, fb.d_toff.p, 0, ns, off);
  galerkin_tiles(c, coarse_columns(c, off - ns), fb, tiles.p, s);
  auto get = [&](int64_t r, int64_t q) {  // entry (r, q), r >= q, of the tile storage
    const int64_t I = r / kTile, J = q / kTile;
    return ((I * (I + 1) / 2 + J) * kTileElems) + (r % kTile) * kTile + (q % kTile);
  };
  std::vector<double> host = tiles.download(s);
  std::vector<double> diag(nh);
  for (int64_t h = 0; h < nh; ++h) diag[h] = host[get(off + h, off + h)];
  if (off > 0) {
    const int npiv = (int)(off / kTile);
    DevBuf<int32_t> dn;
    dn.upload(std::vector<int32_t>{npiv}, s);
    DevBuf<int64_t> dtoff;
    dtoff.upload(std::vector<int64_t>{0, (int64_t)fb.nt[0]}, s);
    DevBuf<double> dinv;
    dinv.alloc((int64_t)fb.nt[0] * kTileElems);
    chol_factor(fb, tiles.p, dn.p, npiv, dinv.p, dtoff.p, c->d_err.p, s);
    check_device_error(c, s);
    host = tiles.download(s);
  }
  std::vector<double> S(nh * nh);
  for (int64_t i = 0; i < nh; ++i)
    for (int64_t j = 0; j <= i; ++j) S[i * nh + j] = S[j * nh + i] = host[get(off + i, off + j)];
  apply_geneo_keep(c, ordered_drop(S, diag, nh, kDepTol));
}

// Z without the dropped GenEO columns
static void apply_geneo_keep(geneo_ctx *c, const std::vector<int64_t> &keep) {
  const int64_t ns = c->n0_snk, nh = c->n0_geneo;
  if ((int64_t)keep.size() == nh) return;
  std::vector<int64_t> ptr(c->zc_ptr.begin(), c->zc_ptr.begin() + ns + 1);
  std::vector<int32_t> row(c->zc_row.begin(), c->zc_row.begin() + c->zc_ptr[ns]);
  std::vector<double> val(c->zc_val.begin(), c->zc_val.begin() + c->zc_ptr[ns]);
  std::vector<int32_t> gs;
  std::vector<double> gl;
  for (int64_t h : keep) {
    const int64_t a = ns + h;
    row.insert(row.end(), c->zc_row.begin() + c->zc_ptr[a], c->zc_row.begin() + c->zc_ptr[a + 1]);
    val.insert(val.end(), c->zc_val.begin() + c->zc_ptr[a], c->zc_val.begin() + c->zc_ptr[a + 1]);
    ptr.push_back((int64_t)row.size());
    gs.push_back(c->geneo_sub[h]);
    gl.push_back(c->geneo_lambda[h]);
  }
  c->zc_ptr = ptr;
  c->zc_row = row;
  c->zc_val = val;
  c->geneo_sub = gs;
  c->geneo_lambda = gl;
  c->n0_geneo = (int64_t)keep.size();
  c->n0 = ns + c->n0_geneo;
}

// Independent components: union-find over active cells sharing a vertex;
// an unknown belongs to the component of its lowest containing cell.
static void build_components(geneo_ctx *c) {
  const Topology &t = c->topo;
  const int nx = t.nx, ny = t.ny, nz = t.nz;
  std::vector<int32_t> par(t.ncells, -1);
  for (int32_t cl : t.cells) par[cl] = cl;
  std::function<int32_t(int32_t)> find = [&](int32_t a) {
    while (par[a] != a) {
      par[a] = par[par[a]];
      a = par[a];
    }
    return a;
  };
  for (int32_t cl : t.cells) {
    const int i = cl % nx, j = (cl / nx) % ny, k = cl / (nx * ny);
    for (int dk = 0; dk <= 1; ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          if (dk == 0 && (dj < 0 || (dj == 0 && di <= 0))) continue;  // each pair once
          const int a = i + di, b = j + dj, d = k + dk;
          if (a < 0 || b < 0 || a >= nx || b >= ny || d >= nz) continue;
          const int32_t o = a + nx * (b + ny * d);
          if (par[o] < 0) continue;
          const int32_t ra = find(cl), rb = find(o);
          if (ra != rb) par[std::max(ra, rb)] = std::min(ra, rb);
        }
  }
  const int64_t n = t.ndofs();
  std::vector<int32_t> comp_id(t.ncells, -1), seg(n);
  int32_t ncomp = 0;
  c->seg_ok = true;
  for (int64_t e = 0; e < n; ++e) {
    const int32_t r = find(t.first_cell[t.dof_edge[e]]);
    if (comp_id[r] < 0) comp_id[r] = ncomp++;
    seg[e] = comp_id[r];
    if (e > 0 && seg[e] < seg[e - 1]) c->seg_ok = false;
  }
  c->seg_off.assign(1, 0);
  if (c->seg_ok) {
    for (int64_t e = 1; e <= n; ++e)
      if (e == n || seg[e] != seg[e - 1]) c->seg_off.push_back(e);
    if ((int64_t)c->seg_off.size() != ncomp + 1) c->seg_ok = false;
  }
  if (!c->seg_ok) c->seg_off.clear();
  c->seg_of = std::move(seg);
}

void setup_topology(geneo_ctx *c) {
  Topology &t = c->topo;
  build_topology(c->nx, c->ny, c->nz, c->h, c->active.data(), t,
                 c->natural.empty() ? nullptr : c->natural.data());
  if (t.ndofs() == 0) throw Error(GENEO_ERR_INVALID_ARG, "the mesh has no interior edge");
  build_decomposition(t, c->px, c->py, c->pz, c->overlap, c->dec,
                      c->cell_part.empty() ? nullptr : c->cell_part.data());
  build_components(c);
  build_local_structure(t, c->dec, c->ls);
  if (c->host_only && c->opt.coarse != GENEO_COARSE_NONE) {
    if (c->opt.coarse == GENEO_COARSE_NK) build_nk(t, c->snk);
    else build_snk(t, c->dec, c->snk);
    c->n0 = c->n0_snk = (int64_t)c->snk.sub.size();
    c->zc_ptr = c->snk.ptr;
    c->zc_row = c->snk.row;
    c->zc_val.assign(c->snk.sgn.begin(), c->snk.sgn.end());
  }
}

void setup_all(geneo_ctx *c) {
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = c->stream;
  Topology &t = c->topo;
  setup_topology(c);
  c->d_seg_of.upload(c->seg_of, s);
  if (c->seg_ok) c->d_seg_off.upload(c->seg_off, s);
  c->d_err.alloc(1);
  c->d_err.zero(s);

  // --- global matrix
  const int64_t nt = t.ntets(), n = t.ndofs();
  c->d_tets.upload(t.tets, s);
  c->d_tet_cell.upload(t.tet_cell, s);
  c->d_tet_edges.upload(t.tet_edges, s);
  {
    std::vector<int32_t> tail(t.nedges());
    for (int64_t e = 0; e < t.nedges(); ++e) tail[e] = t.edges[2 * e];
    c->d_edge_tail.upload(tail, s);
    c->d_edge_dir.upload(t.edge_dir, s);
  }
  c->d_mu.upload(c->mu_inv, s);
  c->d_eps.upload(c->eps, s);
  c->d_Ae.alloc(nt * 36);
  k_element<<<grid_for(nt, 128), 128, 0, s>>>(c->d_tets.p, c->d_tet_cell.p, c->d_mu.p, c->d_eps.p,
                                              c->gamma, c->nx, c->ny, c->h[0], c->h[1], c->h[2],
                                              nt, c->d_Ae.p);
  GENEO_CHECK_LAUNCH();
  c->d_rowptr.upload(t.rowptr, s);
  c->d_col.upload(t.col, s);
  c->d_cptr.upload(t.cptr, s);
  c->d_cidx.upload(t.cidx, s);
  c->d_rptr.upload(t.rptr, s);
  c->d_ridx.upload(t.ridx, s);
  c->d_val.alloc(t.nnz());
  k_gather_sum<<<grid_for(t.nnz(), 256), 256, 0, s>>>(c->d_cptr.p, c->d_cidx.p, c->d_Ae.p,
                                                      t.nnz(), c->d_val.p);
  GENEO_CHECK_LAUNCH();
  build_sell(c, s);

  auto last = t0;
  auto stage_mark = [&](int k) {
    GENEO_CUDA(cudaStreamSynchronize(s));
    const auto now = std::chrono::steady_clock::now();
    if (k == 0) c->stage_s[0] = std::chrono::duration<double>(now - t0).count();
    else c->stage_s[k] = std::chrono::duration<double>(now - last).count();
    last = now;
  };
  stage_mark(0);
  // --- local factors: A_i extracted into tile-packed storage and inverted
  const Decomposition &d = c->dec;
  std::vector<int64_t> dims(d.nsub);
  for (int i = 0; i < d.nsub; ++i) dims[i] = d.ni(i);
  c->loc.layout(dims);
  c->loc.upload_meta(s);
  c->loc_f64.alloc(tile_elems(c->loc));
  tiles_init_padding(c->loc, c->loc_f64.p, s);
  {
    DevBuf<int64_t> noff, lrp, ncp;
    DevBuf<int32_t> lcol, lpos;
    noff.upload(d.N_off, s);
    lrp.upload(c->ls.lrowptr, s);
    lcol.upload(c->ls.lcol, s);
    lpos.upload(c->ls.lpos, s);
    k_extract_local<<<dim3(64, d.nsub), 256, 0, s>>>(noff.p, lrp.p, lcol.p, lpos.p, c->d_val.p,
                                                     c->loc.d_toff.p, c->loc_f64.p);
    GENEO_CHECK_LAUNCH();
  }
  c->loc.schedule(c->sm_count, s);
  {
    std::vector<int32_t> l2g(c->loc.vlen, -1);
    std::vector<int64_t> g2l(c->ls.g2l_slot.size());
    std::vector<int64_t> slot_pad(d.N_off[d.nsub]);
    for (int i = 0; i < d.nsub; ++i)
      for (int64_t r = 0; r < d.ni(i); ++r) {
        slot_pad[d.N_off[i] + r] = c->loc.voff[i] + r;
        l2g[c->loc.voff[i] + r] = d.N_idx[d.N_off[i] + r];
      }
    for (size_t k = 0; k < g2l.size(); ++k) g2l[k] = slot_pad[c->ls.g2l_slot[k]];
    c->d_l2g.upload(l2g, s);
    c->d_g2l_ptr.upload(c->ls.g2l_ptr, s);
    c->d_g2l.upload(g2l, s);
  }
  // optional gradient shift A_j -> A_j (I + rho xi_j), then the explicit inverses
  if (c->opt.gradient_shift) apply_gradient_shift(c);
  {
    DevBuf<double> ws;
    ws.alloc(spd_workspace_elems(c->loc));
    spd_invert(c->loc, c->loc_f64.p, ws.p, c->d_err.p, s);
    check_device_error(c, s);
  }
  stage_mark(1);
  if (c->opt.precision == GENEO_PREC_FP32 || c->opt.precision == GENEO_PREC_BF16) {
    build_split_factors(c);
    c->local_prec = GENEO_PREC_FP32;
  }
  if (c->opt.precision == GENEO_PREC_BF16) {
    build_bf16_factors(c);
    c->local_prec = GENEO_PREC_BF16;
  }

  stage_mark(2);
  // the SYMV autotuner runs before the eigensolves, which apply the local
  // factors every LOBPCG iteration
  if (c->opt.autotune) autotune_symv(c);
  stage_mark(6);
  // --- coarse space
  c->n0 = c->n0_snk = c->n0_geneo = 0;
  if (c->opt.coarse != GENEO_COARSE_NONE) {
    // near-kernel part of Z: split (SNK, the method) or global (NK, Sec. 4)
    if (c->opt.coarse == GENEO_COARSE_NK) build_nk(t, c->snk);
    else build_snk(t, d, c->snk);
    c->n0_snk = (int64_t)c->snk.sub.size();
    c->zc_ptr = c->snk.ptr;
    c->zc_row = c->snk.row;
    c->zc_val.resize(c->snk.sgn.size());
    for (size_t k = 0; k < c->snk.sgn.size(); ++k) c->zc_val[k] = (double)c->snk.sgn[k];
    c->n0 = c->n0_snk;
  }
  if (c->zc_ptr.empty()) c->zc_ptr.push_back(0);
  if (c->opt.geneo) {
    if (c->opt.warm_start || c->opt.keep_eigvecs) {
      if (!c->xi) {
        c->xi.reset(new XiOp());
        build_xi_operator(c, *c->xi, s);
      }
      build_mlp_features(c);
    }
    geneo_eigenvectors(c);  // appends GenEO candidates to zc_* and sets n0_geneo
    stage_mark(3);
    if (c->n0_geneo > 0) {
      if (c->opt.coarse_dense) geneo_filter(c);
      else geneo_filter_mf(c);
    }
    stage_mark(4);
  }
  if (c->n0 > 0 && !c->opt.coarse_dense) {
    build_z_csr(c);
    mf_setup(c);
    c->crs_x.alloc(c->n0);
    c->crs_y.alloc(c->n0);
    c->crs_x.zero(s);
    if (c->opt.autotune) autotune_coarse(c);
  } else if (c->n0 > 0) {
    build_z_csr(c);
    c->crs.layout({c->n0});
    c->crs.upload_meta(s);
    c->crs_f64.alloc(tile_elems(c->crs));
    tiles_init_padding(c->crs, c->crs_f64.p, s);
    galerkin_tiles(c, coarse_columns(c, 0), c->crs, c->crs_f64.p, s);
    DevBuf<double> ws;
    ws.alloc(spd_workspace_elems(c->crs));
    spd_invert(c->crs, c->crs_f64.p, ws.p, c->d_err.p, s);
    check_device_error(c, s);
    c->crs.schedule(c->sm_count, s);
    c->crs_x.alloc(c->crs.vlen);
    c->crs_y.alloc(c->crs.vlen);
    c->crs_x.zero(s);
  }

  stage_mark(5);
  // --- work vectors (one right-hand side; grown on demand)
  for (auto *v : {&c->h_b, &c->h_x}) v->alloc(n);
  reserve_rhs(c, 1);
  check_device_error(c, s);
  c->setup_seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  c->stage_s[7] = c->setup_seconds;
}

void assemble_rhs(geneo_ctx *c, const double *fslot_host, double *b, cudaStream_t s) {
  const Topology &t = c->topo;
  const int64_t ne = t.nedges(), nt = t.ntets();
  DevBuf<double> fs, ce, mc;
  fs.alloc(t.nverts * 21);
  GENEO_CUDA(cudaMemcpyAsync(fs.p, fslot_host, sizeof(double) * t.nverts * 21,
                             cudaMemcpyHostToDevice, s));
  ce.alloc(ne);
  mc.alloc(nt * 6);
  k_rhs_edge<<<grid_for(ne, 256), 256, 0, s>>>(fs.p, c->d_edge_tail.p, c->d_edge_dir.p, c->h[0],
                                               c->h[1], c->h[2], ne, ce.p);
  k_rhs_element<<<grid_for(nt, 128), 128, 0, s>>>(c->d_tets.p, c->d_tet_edges.p, ce.p, c->nx,
                                                  c->ny, c->h[0], c->h[1], c->h[2], nt, mc.p);
  k_gather_sum<<<grid_for(t.ndofs(), 256), 256, 0, s>>>(c->d_rptr.p, c->d_ridx.p, mc.p,
                                                        t.ndofs(), b);
  GENEO_CHECK_LAUNCH();
  GENEO_CUDA(cudaStreamSynchronize(s));  // temporaries are freed on return
}

}  // namespace geneo
