// Sparse direct coarse solve: multifrontal Cholesky of E = Z^T A Z (Sec. 2).
//
// Ordering: geometric nested dissection on the vertex coordinates of the
// split near-kernel columns.  Column (i, v) couples only with columns whose
// vertices share a tetrahedron with v, so a plane of vertices separates the
// two half-boxes; regions of at most `leaf` columns (256 by default) become leaf fronts and the
// GenEO columns (dense couplings inside their subdomain) are eliminated last,
// in the root front.  Symbolic factorisation on the host: front f holds its
// pivots P_f (consecutive in the elimination order, padded to a tile
// multiple) followed by its update rows U_f.  Numeric factorisation on the
// GPU, one tree level at a time: the entries of E are scattered into the
// fronts, children's Schur complements are extend-added into their parents
// (one child slot per launch, so no two writes collide), and the pivot tiles
// are factored by the tiled Cholesky (the trailing tiles then hold the Schur
// complement).  The pivot blocks are finally inverted, so a solve is a
// sequence of dense tile GEMVs per level: forward y_P = L11^-1 w_P and
// w_U -= L21 y_P (passed to the parent), backward t_P = y_P - L21^T x_U and
// x_P = L11^-T t_P.
#include <algorithm>
#include <numeric>

#include "setup.hpp"

namespace geneo {

namespace {
constexpr int kLeafDefault = 256;
constexpr int kChunk = 4;  // tiles per task of the solve's tile GEMVs

struct Front {
  std::vector<int32_t> cols;      // pivot columns (coarse column ids)
  std::vector<int32_t> children;
  int parent = -1;
  int level = 0;
  int64_t first = 0;              // elimination position of the first pivot
  int npiv = 0, npivp = 0;        // pivots, padded to a tile multiple
  std::vector<int64_t> upd;       // update rows (elimination positions, ascending)
};

void nd_build(const std::vector<int32_t> &cols, const std::vector<int32_t> &coord, int lo[3],
              int hi[3], int leaf, std::vector<Front> &F, std::vector<int> &roots) {
  if ((int)cols.size() <= leaf) {
    if (cols.empty()) return;
    Front f;
    f.cols = cols;
    F.push_back(f);
    roots.push_back((int)F.size() - 1);
    return;
  }
  int axis = 0;
  for (int a = 1; a < 3; ++a)
    if (hi[a] - lo[a] > hi[axis] - lo[axis]) axis = a;
  if (hi[axis] <= lo[axis]) {  // a single vertex holding many columns
    Front f;
    f.cols = cols;
    F.push_back(f);
    roots.push_back((int)F.size() - 1);
    return;
  }
  const int s = (lo[axis] + hi[axis]) / 2;
  std::vector<int32_t> left, sep, right;
  for (int32_t c : cols) {
    const int x = coord[3 * c + axis];
    (x < s ? left : (x == s ? sep : right)).push_back(c);
  }
  std::vector<int> sub;
  int l2[3] = {lo[0], lo[1], lo[2]}, h2[3] = {hi[0], hi[1], hi[2]};
  h2[axis] = s - 1;
  nd_build(left, coord, lo, h2, leaf, F, sub);
  l2[axis] = s + 1;
  nd_build(right, coord, l2, hi, leaf, F, sub);
  if (sep.empty()) {
    roots.insert(roots.end(), sub.begin(), sub.end());
    return;
  }
  Front f;
  f.cols = sep;
  f.children = sub;
  F.push_back(f);
  const int id = (int)F.size() - 1;
  for (int ch : sub) F[ch].parent = id;
  roots.push_back(id);
}

__global__ void k_scatter(const double *__restrict__ vals, const int64_t *__restrict__ off1,
                          const int64_t *__restrict__ off2, int64_t nq, double *__restrict__ data) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  data[off1[q]] = vals[q];
  if (off2[q] >= 0) data[off2[q]] = vals[q];
}

__global__ void k_set_rows_identity(double *data, const int64_t *__restrict__ diag_off, int64_t n) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q < n) data[diag_off[q]] = 1.0;
}

// parent += child's update block; one CTA per (child, tile of its U block)
__global__ void k_extend_add(const int32_t *__restrict__ it_child, const int32_t *__restrict__ it_I,
                             const int32_t *__restrict__ it_J, const int32_t *__restrict__ parent,
                             const int32_t *__restrict__ npivp, const int64_t *__restrict__ nupd,
                             const int64_t *__restrict__ map_off, const int32_t *__restrict__ map,
                             const int64_t *__restrict__ toff, double *__restrict__ data) {
  const int c = it_child[blockIdx.x], I = it_I[blockIdx.x], J = it_J[blockIdx.x];
  const int p = parent[c];
  const int64_t nu = nupd[c];
  const double *src = data + (toff[c] + (int64_t)I * (I + 1) / 2 + J) * kTileElems;
  for (int e = threadIdx.x; e < kTileElems; e += blockDim.x) {
    const int64_t li = (int64_t)I * kTile + (e >> 6) - npivp[c];
    const int64_t lj = (int64_t)J * kTile + (e & 63) - npivp[c];
    if (li < 0 || lj < 0 || li >= nu || lj >= nu || lj > li) continue;
    const int64_t P = map[map_off[c] + li], Q = map[map_off[c] + lj];
    const int PI = (int)(P / kTile), QI = (int)(Q / kTile);
    const double v = src[e];
    double *t = data + (toff[p] + (int64_t)PI * (PI + 1) / 2 + QI) * kTileElems;
    t[(P % kTile) * kTile + (Q % kTile)] += v;
    if (PI == QI && P != Q) t[(Q % kTile) * kTile + (P % kTile)] += v;
  }
}

// forward gather: w[f][l] = c(pivot l) + sum of children's update entries
__global__ void k_mf_gather(const int32_t *__restrict__ rf, const int32_t *__restrict__ rl,
                            const int64_t *__restrict__ gptr, const int64_t *__restrict__ gidx,
                            const int64_t *__restrict__ first, const int32_t *__restrict__ npiv,
                            const int64_t *__restrict__ voff, int64_t nrows, int64_t n0,
                            int64_t vlen, const double *__restrict__ cpos,
                            double *__restrict__ w) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nrows) return;
  cpos += blockIdx.y * n0;  // right-hand side blockIdx.y
  w += blockIdx.y * vlen;
  const int f = rf[q], l = rl[q];
  double v = l < npiv[f] ? cpos[first[f] + l] : 0.0;
  for (int64_t k = gptr[q]; k < gptr[q + 1]; ++k) v += w[gidx[k]];
  w[voff[f] + l] = v;
}

// One task of a tile GEMV phase: tiles j0 <= K < j1 of tile row I (row
// modes) or tile column I (column modes) of front f.  Tasks of one output
// tile are consecutive (slots rbase .. rbase + nch - 1) and share counter cnt.
struct MfTask {
  int32_t f, I, j0, j1;
  int32_t slot, rbase, nch, cnt;
};

// Phases of the solve (T = tiles of front f, v = input, o = output tile):
//   0: y_I  = sum_{J<=I} Y(I,J) w_J            (forward, pivot rows)
//   1: w_I -= sum_{J<npivt} L(I,J) y_J          (forward, update rows)
//   2: t_J  = y_J - sum_{I>=npivt} L(I,J)^T x_I (backward, x_I gathered from the
//                                                solution at the update rows)
//   3: x_J  = sum_{J<=I<npivt} Y(I,J)^T t_I      (backward, to the solution)
// Each task reduces its tiles to a 64-vector; a task whose output tile has
// several tasks stores it to part[slot] and the last of them to finish sums
// the stored vectors in slot order (deterministic) and writes the output.
struct MfArgs {
  const int32_t *npivt, *npiv, *npivp;
  const int64_t *nupd, *first, *uoff, *upos, *toff, *voff;
  const double *T;
  double *wbuf, *ybuf, *tbuf, *xpos, *part;
  int32_t *cnt;
  // right-hand sides: k columns, column strides of the buffers above
  int k;
  int64_t ldv, ldx, ldp, ldc;
};

// blockIdx.x = task * k + column: the k columns of a task run in adjacent
// CTAs, so its tiles are read from DRAM once and from L2 for the others
template <int kMode>
__global__ void __launch_bounds__(256) k_mf_tiles(const MfTask *__restrict__ tasks, MfArgs a) {
  const MfTask tk = tasks[blockIdx.x / a.k];
  {
    const int64_t col = blockIdx.x % a.k;
    a.wbuf += col * a.ldv;
    a.ybuf += col * a.ldv;
    a.tbuf += col * a.ldv;
    a.xpos += col * a.ldx;
    a.part += col * a.ldp;
    a.cnt += col * a.ldc;
  }
  const int f = tk.f, O = tk.I;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __shared__ double red[8][kTile];
  __shared__ double vec[kTile];
  __shared__ int last;
  const int64_t vo = a.voff[f];
  const int nk = tk.j1 - tk.j0;  // tiles of this task, at most kChunk
  if (kMode <= 1) {
    // row modes: warp w owns rows 8w..8w+7, lane l columns 2l, 2l+1.  All of
    // the task's tiles are loaded (predicated) before the first use, so
    // their DRAM latencies overlap
    const double *vin = kMode == 0 ? a.wbuf : a.ybuf;
    double2 v[kChunk][8], x[kChunk];
#pragma unroll
    for (int q = 0; q < kChunk; ++q) {
      const int K = tk.j0 + q;
      if (q < nk) {
        const double *t = a.T + (a.toff[f] + (int64_t)O * (O + 1) / 2 + K) * kTileElems;
        x[q] = *reinterpret_cast<const double2 *>(vin + vo + (int64_t)K * kTile + 2 * l);
#pragma unroll
        for (int r = 0; r < 8; ++r)
          v[q][r] = __ldg(reinterpret_cast<const double2 *>(t + (w * 8 + r) * kTile + 2 * l));
      }
    }
    double acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = 0.0;
#pragma unroll
    for (int q = 0; q < kChunk; ++q)
      if (q < nk)
#pragma unroll
        for (int r = 0; r < 8; ++r) acc[r] = fma(v[q][r].x, x[q].x, fma(v[q][r].y, x[q].y, acc[r]));
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      double vv = acc[r];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) vv += __shfl_xor_sync(0xffffffffu, vv, o);
      if (l == 0) vec[w * 8 + r] = vv;
    }
  } else {
    // column modes: warp w owns rows 8w..8w+7 of every tile, lane l columns
    // 2l, 2l+1.  The input entries of the task's rows are staged in shared
    // memory first (phase 2 gathers them through the update-row map, all in
    // parallel), and the tiles are loaded (predicated) before the first use
    __shared__ double xs[kChunk * kTile];
    for (int e = threadIdx.x; e < nk * kTile; e += blockDim.x) {
      const int64_t row = (int64_t)tk.j0 * kTile + e;
      double xv;
      if (kMode == 2) {
        const int64_t u = row - a.npivp[f];
        xv = (u >= 0 && u < a.nupd[f]) ? a.xpos[a.upos[a.uoff[f] + u]] : 0.0;
      } else {
        xv = a.tbuf[vo + row];
      }
      xs[e] = xv;
    }
    double2 v[kChunk][8];
#pragma unroll
    for (int q = 0; q < kChunk; ++q) {
      const int K = tk.j0 + q;
      if (q < nk) {
        const double *t = a.T + (a.toff[f] + (int64_t)K * (K + 1) / 2 + O) * kTileElems;
#pragma unroll
        for (int r = 0; r < 8; ++r)
          v[q][r] = __ldg(reinterpret_cast<const double2 *>(t + (w * 8 + r) * kTile + 2 * l));
      }
    }
    __syncthreads();
    double c0 = 0.0, c1 = 0.0;
#pragma unroll
    for (int q = 0; q < kChunk; ++q)
      if (q < nk)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const double xv = xs[q * kTile + w * 8 + r];
          c0 = fma(v[q][r].x, xv, c0);
          c1 = fma(v[q][r].y, xv, c1);
        }
    red[w][2 * l] = c0;
    red[w][2 * l + 1] = c1;
    __syncthreads();
    if (threadIdx.x < kTile) {
      double vv = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) vv += red[q][threadIdx.x];
      vec[threadIdx.x] = vv;
    }
  }
  __syncthreads();
  if (tk.nch > 1) {
    if (threadIdx.x < kTile) {
      a.part[(int64_t)tk.slot * kTile + threadIdx.x] = vec[threadIdx.x];
      __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      last = atomicAdd(&a.cnt[tk.cnt], 1) == tk.nch - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < kTile) {
      double v = 0.0;
      for (int k = 0; k < tk.nch; ++k) v += __ldcg(a.part + (int64_t)(tk.rbase + k) * kTile + threadIdx.x);
      vec[threadIdx.x] = v;
    }
    if (threadIdx.x == 0) a.cnt[tk.cnt] = 0;
    __syncthreads();
  }
  if (threadIdx.x < kTile) {
    const int64_t idx = (int64_t)O * kTile + threadIdx.x;
    const double v = vec[threadIdx.x];
    if (kMode == 0) a.ybuf[vo + idx] = v;
    else if (kMode == 1) a.wbuf[vo + idx] -= v;
    else if (kMode == 2) a.tbuf[vo + idx] = a.ybuf[vo + idx] - v;
    else if (idx < a.npiv[f]) a.xpos[a.first[f] + idx] = v;
  }
}

__global__ void k_perm(const int64_t *__restrict__ idx, const double *__restrict__ src,
                       double *__restrict__ dst, int64_t n, int to_pos) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= n) return;
  src += blockIdx.y * n;
  dst += blockIdx.y * n;
  if (to_pos) dst[idx[a]] = src[a];
  else dst[a] = src[idx[a]];
}

}  // namespace

struct MfLevel {
  int max_npivt = 0;
  DevBuf<int32_t> npiv_lvl;                         // per front: pivot tiles if in level
  std::vector<DevBuf<int32_t>> ea_child, ea_I, ea_J;  // extend-add items per child slot
  std::vector<int> ea_n;
  DevBuf<int32_t> rf, rl;                           // gather rows
  DevBuf<int64_t> gptr, gidx;
  int64_t nrows = 0;
  DevBuf<MfTask> task[4];                           // tile GEMV tasks per phase
  int ntask[4] = {0, 0, 0, 0};
};

struct Multifrontal {
  int nfront = 0;
  TileBatch fb;
  DevBuf<double> L, Y, dinv, wbuf, ybuf, tbuf, cpos, xpos, part;  // solve buffers: kcap columns
  DevBuf<int32_t> cnt;
  int kcap = 0, nslot = 0, ncnt = 0;
  DevBuf<int64_t> dtoff, first, nupd, uoff, upos, pos;
  DevBuf<int32_t> npiv, npivp, npivt, parent, nt;
  std::vector<MfLevel> levels;
  int64_t factor_bytes = 0;
  int64_t solve_tiles = 0;  // factor tiles one solve reads (all phases, all levels)
};

void MfDeleter::operator()(Multifrontal *m) const { delete m; }

void mf_setup(geneo_ctx *c, MfSchur *schur) {
  cudaStream_t s = c->stream;
  const int64_t n0 = c->n0;
  const Topology &t = c->topo;
  auto M = new Multifrontal();
  c->mf.reset(M);
  // --- nested dissection on vertex coordinates
  std::vector<int32_t> coord(3 * n0, 0), snkcols, geneo;
  int lo[3] = {0, 0, 0}, hi[3] = {t.nx, t.ny, t.nz};
  for (int64_t a = 0; a < n0; ++a) {
    if (a < c->n0_snk) {
      const int64_t v = c->snk.vert[a];
      coord[3 * a] = (int32_t)(v % (t.nx + 1));
      coord[3 * a + 1] = (int32_t)((v / (t.nx + 1)) % (t.ny + 1));
      coord[3 * a + 2] = (int32_t)(v / ((int64_t)(t.nx + 1) * (t.ny + 1)));
      snkcols.push_back((int32_t)a);
    } else {
      geneo.push_back((int32_t)a);
    }
  }
  std::vector<Front> F;
  std::vector<int> roots;
  nd_build(snkcols, coord, lo, hi, c->opt.coarse_leaf > 0 ? c->opt.coarse_leaf : kLeafDefault, F,
           roots);
  if (!geneo.empty() || roots.empty()) {
    Front f;
    f.cols = geneo;
    f.children = roots;
    F.push_back(f);
    const int id = (int)F.size() - 1;
    for (int ch : roots) F[ch].parent = id;
    roots.assign(1, id);
  }
  // --- postorder positions
  std::vector<int> order;
  {
    std::vector<std::pair<int, int>> st;
    for (int r : roots) st.push_back({r, 0});
    std::reverse(st.begin(), st.end());
    while (!st.empty()) {
      auto &top = st.back();
      const int f = top.first;
      if (top.second < (int)F[f].children.size()) {
        const int ch = F[f].children[top.second++];
        st.push_back({ch, 0});
      } else {
        order.push_back(f);
        st.pop_back();
      }
    }
  }
  std::vector<int64_t> pos(n0, -1);
  std::vector<int32_t> front_of(n0, -1);
  int64_t next = 0;
  for (int f : order) {
    F[f].first = next;
    for (int32_t a : F[f].cols) {
      pos[a] = next++;
      front_of[pos[a]] = f;
    }
    F[f].npiv = (int)F[f].cols.size();
    F[f].npivp = (F[f].npiv + kTile - 1) / kTile * kTile;
    int lv = 0;
    for (int ch : F[f].children) lv = std::max(lv, F[ch].level + 1);
    F[f].level = lv;
  }
  if (next != n0) throw Error(GENEO_ERR_CUDA, "internal: coarse ordering incomplete");
  // --- Galerkin pattern in elimination order, upper adjacency
  Columns X;
  for (int64_t a = 0; a < n0; ++a) {
    for (int64_t k = c->zc_ptr[a]; k < c->zc_ptr[a + 1]; ++k) {
      X.row.push_back(c->zc_row[k]);
      X.val.push_back(c->zc_val[k]);
    }
    X.ptr.push_back((int64_t)X.row.size());
    X.mat.push_back(0);
    X.loc.push_back((int32_t)pos[a]);
  }
  GalerkinPlan P;
  galerkin_plan(c, X, P, s);
  std::vector<std::vector<int64_t>> up(n0);
  for (int64_t a = 0; a < n0; ++a)
    for (int64_t q = P.pptr[a]; q < P.pptr[a + 1]; ++q) {
      const int64_t b = P.pcol[q];
      if (b != a) up[pos[b]].push_back(pos[a]);
    }
  // --- symbolic: update rows of every front (postorder)
  std::vector<uint8_t> mark(n0, 0);
  for (int f : order) {
    Front &fr = F[f];
    const int64_t last = fr.first + fr.npiv - 1;
    std::vector<int64_t> S;
    for (int64_t p = fr.first; p <= last; ++p)
      for (int64_t qpos : up[p])
        if (qpos > last && !mark[qpos]) {
          mark[qpos] = 1;
          S.push_back(qpos);
        }
    for (int ch : fr.children)
      for (int64_t qpos : F[ch].upd)
        if (qpos > last && !mark[qpos]) {
          mark[qpos] = 1;
          S.push_back(qpos);
        }
    for (int64_t qpos : S) mark[qpos] = 0;
    std::sort(S.begin(), S.end());
    fr.upd = S;
  }
  const int nf = (int)F.size();
  M->nfront = nf;
  auto local = [&](int f, int64_t x) -> int64_t {
    const Front &fr = F[f];
    if (x >= fr.first && x < fr.first + fr.npiv) return x - fr.first;
    auto it = std::lower_bound(fr.upd.begin(), fr.upd.end(), x);
    if (it == fr.upd.end() || *it != x) return -1;
    return fr.npivp + (it - fr.upd.begin());
  };
  std::vector<int64_t> dims(nf);
  for (int f = 0; f < nf; ++f) dims[f] = std::max<int64_t>(1, F[f].npivp + (int64_t)F[f].upd.size());
  M->fb.layout(dims);
  M->fb.upload_meta(s);
  TileBatch &fb = M->fb;
  M->L.alloc(tile_elems(fb));
  tiles_init_padding(fb, M->L.p, s);
  auto elem = [&](int f, int64_t r, int64_t q) {  // r >= q
    const int64_t I = r / kTile, J = q / kTile;
    return (fb.toff[f] + I * (I + 1) / 2 + J) * kTileElems + (r % kTile) * kTile + (q % kTile);
  };
  {
    // identity on the pivot padding rows
    std::vector<int64_t> pad;
    for (int f = 0; f < nf; ++f)
      for (int64_t r = F[f].npiv; r < F[f].npivp; ++r) pad.push_back(elem(f, r, r));
    DevBuf<int64_t> dp;
    dp.upload(pad, s);
    if (dp.n) k_set_rows_identity<<<grid_for(dp.n, 256), 256, 0, s>>>(M->L.p, dp.p, dp.n);
    // entries of E into the front eliminating the lower-positioned column
    const int64_t nq = (int64_t)P.pcol.size();
    std::vector<int64_t> o1(nq), o2(nq);
    for (int64_t a = 0; a < n0; ++a)
      for (int64_t q = P.pptr[a]; q < P.pptr[a + 1]; ++q) {
        const int64_t b = P.pcol[q];
        const int f = front_of[pos[b]];
        const int64_t la = local(f, pos[a]), lb = local(f, pos[b]);
        if (la < 0 || lb < 0 || la < lb) throw Error(GENEO_ERR_CUDA, "internal: coarse symbolic");
        o1[q] = elem(f, la, lb);
        o2[q] = (la / kTile == lb / kTile && la != lb)
                    ? (fb.toff[f] + (la / kTile) * (la / kTile + 1) / 2 + la / kTile) * kTileElems +
                          (lb % kTile) * kTile + (la % kTile)
                    : -1;
      }
    DevBuf<double> vals;
    vals.alloc(nq);
    galerkin_values(P, vals.p, s);
    DevBuf<int64_t> d1, d2;
    d1.upload(o1, s);
    d2.upload(o2, s);
    k_scatter<<<grid_for(nq, 256), 256, 0, s>>>(vals.p, d1.p, d2.p, nq, M->L.p);
    GENEO_CHECK_LAUNCH();
    GENEO_CUDA(cudaStreamSynchronize(s));
    if (schur) {
      // diagonal of E on the GenEO columns (pattern entry (a, a))
      const std::vector<double> hv = vals.download(s);
      const int64_t ns = c->n0_snk;
      schur->nh = n0 - ns;
      schur->diag.assign(schur->nh, 0.0);
      for (int64_t a = ns; a < n0; ++a)
        for (int64_t q = P.pptr[a]; q < P.pptr[a + 1]; ++q)
          if (P.pcol[q] == a) schur->diag[a - ns] = hv[q];
    }
  }
  // --- per-front metadata on the device
  std::vector<int32_t> h_npiv(nf), h_npivp(nf), h_npivt(nf), h_parent(nf);
  std::vector<int64_t> h_first(nf), h_nupd(nf), h_uoff(nf + 1, 0), h_upos, h_dtoff(nf + 1, 0);
  std::vector<int64_t> h_mapoff(nf + 1, 0);
  std::vector<int32_t> h_map;
  for (int f = 0; f < nf; ++f) {
    h_npiv[f] = F[f].npiv;
    h_npivp[f] = F[f].npivp;
    h_npivt[f] = F[f].npivp / kTile;
    h_parent[f] = F[f].parent;
    h_first[f] = F[f].first;
    h_nupd[f] = (int64_t)F[f].upd.size();
    h_upos.insert(h_upos.end(), F[f].upd.begin(), F[f].upd.end());
    h_uoff[f + 1] = (int64_t)h_upos.size();
    h_dtoff[f + 1] = h_dtoff[f] + fb.nt[f];
    for (int64_t x : F[f].upd) {
      const int64_t lp = F[f].parent >= 0 ? local(F[f].parent, x) : -1;
      if (F[f].parent >= 0 && lp < 0) throw Error(GENEO_ERR_CUDA, "internal: extend-add map");
      h_map.push_back((int32_t)lp);
    }
    h_mapoff[f + 1] = (int64_t)h_map.size();
  }
  M->npiv.upload(h_npiv, s);
  M->npivp.upload(h_npivp, s);
  M->npivt.upload(h_npivt, s);
  M->parent.upload(h_parent, s);
  M->first.upload(h_first, s);
  M->nupd.upload(h_nupd, s);
  M->uoff.upload(h_uoff, s);
  M->upos.upload(h_upos, s);
  M->dtoff.upload(h_dtoff, s);
  M->nt.upload(fb.nt, s);
  M->pos.upload(pos, s);
  DevBuf<int64_t> d_mapoff;
  DevBuf<int32_t> d_map;
  d_mapoff.upload(h_mapoff, s);
  d_map.upload(h_map, s);
  M->dinv.alloc(h_dtoff[nf] * kTileElems);
  // --- levels
  int nlev = 0;
  for (int f = 0; f < nf; ++f) nlev = std::max(nlev, F[f].level + 1);
  M->levels.resize(nlev);
  int nslot = 0, ncnt = 0;
  std::vector<MfTask> tasks[4];
  for (int lv = 0; lv < nlev; ++lv) {
    MfLevel &Lv = M->levels[lv];
    std::vector<int32_t> np(nf, 0);
    int maxslot = 0;
    for (int f = 0; f < nf; ++f)
      if (F[f].level == lv) {
        np[f] = h_npivt[f];
        Lv.max_npivt = std::max(Lv.max_npivt, np[f]);
        maxslot = std::max(maxslot, (int)F[f].children.size());
      }
    Lv.npiv_lvl.upload(np, s);
    Lv.ea_child.resize(maxslot);
    Lv.ea_I.resize(maxslot);
    Lv.ea_J.resize(maxslot);
    Lv.ea_n.assign(maxslot, 0);
    for (int sl = 0; sl < maxslot; ++sl) {
      std::vector<int32_t> ch, ii, jj;
      for (int f = 0; f < nf; ++f)
        if (F[f].level == lv && sl < (int)F[f].children.size()) {
          const int cf = F[f].children[sl];
          const int t0 = F[cf].npivp / kTile, t1 = fb.nt[cf];
          for (int I = t0; I < t1; ++I)
            for (int J = t0; J <= I; ++J) {
              ch.push_back(cf);
              ii.push_back(I);
              jj.push_back(J);
            }
        }
      Lv.ea_n[sl] = (int)ch.size();
      Lv.ea_child[sl].upload(ch, s);
      Lv.ea_I[sl].upload(ii, s);
      Lv.ea_J[sl].upload(jj, s);
    }
    // solve items
    std::vector<int32_t> rf, rl;
    std::vector<int64_t> gp(1, 0), gi;
    for (int f = 0; f < nf; ++f) {
      if (F[f].level != lv) continue;
      const int64_t dim = F[f].npivp + (int64_t)F[f].upd.size();
      std::vector<std::vector<int64_t>> g(dim);
      for (int ch : F[f].children)
        for (size_t u = 0; u < F[ch].upd.size(); ++u) {
          const int64_t lp = h_map[h_mapoff[ch] + u];
          g[lp].push_back(fb.voff[ch] + F[ch].npivp + (int64_t)u);
        }
      for (int64_t l = 0; l < dim; ++l) {
        rf.push_back(f);
        rl.push_back((int32_t)l);
        gi.insert(gi.end(), g[l].begin(), g[l].end());
        gp.push_back((int64_t)gi.size());
      }
      // tile GEMV tasks: output tile O of front f, input tiles [o0, o1)
      // split into chunks of kChunk tiles
      auto add = [&](int ph, int O, int o0, int o1) {
        const int nch = std::max(1, (o1 - o0 + kChunk - 1) / kChunk);
        M->solve_tiles += std::max(0, o1 - o0);
        const int rbase = nslot;
        for (int k = 0; k < nch; ++k) {
          MfTask tk;
          tk.f = f;
          tk.I = O;
          tk.j0 = o0 + k * kChunk;
          tk.j1 = std::min(o1, o0 + (k + 1) * kChunk);
          tk.slot = nslot++;
          tk.rbase = rbase;
          tk.nch = nch;
          tk.cnt = ncnt;
          tasks[ph].push_back(tk);
        }
        ++ncnt;
      };
      const int npt = h_npivt[f], ntf = fb.nt[f];
      for (int O = 0; O < npt; ++O) add(0, O, 0, O + 1);
      for (int O = npt; O < ntf; ++O) add(1, O, 0, npt);
      // (a front without update rows gets one empty task: t = y)
      for (int O = 0; O < npt; ++O) add(2, O, npt, ntf);
      for (int O = 0; O < npt; ++O) add(3, O, O, npt);
    }
    for (int ph = 0; ph < 4; ++ph) {
      Lv.task[ph].upload(tasks[ph], s);
      Lv.ntask[ph] = (int)tasks[ph].size();
      tasks[ph].clear();
    }
    Lv.rf.upload(rf, s);
    Lv.rl.upload(rl, s);
    Lv.gptr.upload(gp, s);
    Lv.gidx.upload(gi, s);
    Lv.nrows = (int64_t)rf.size();
  }
  M->nslot = std::max(1, nslot);
  M->ncnt = std::max(1, ncnt);
  // --- numeric factorisation, level by level
  for (int lv = 0; lv < nlev; ++lv) {
    MfLevel &Lv = M->levels[lv];
    for (size_t sl = 0; sl < Lv.ea_n.size(); ++sl)
      if (Lv.ea_n[sl])
        k_extend_add<<<Lv.ea_n[sl], 256, 0, s>>>(Lv.ea_child[sl].p, Lv.ea_I[sl].p, Lv.ea_J[sl].p,
                                                  M->parent.p, M->npivp.p, M->nupd.p, d_mapoff.p,
                                                  d_map.p, fb.d_toff.p, M->L.p);
    if (schur && lv == nlev - 1) break;  // the root (GenEO columns) stays unfactored
    if (Lv.max_npivt > 0)
      chol_factor(fb, M->L.p, Lv.npiv_lvl.p, Lv.max_npivt, M->dinv.p, M->dtoff.p, c->d_err.p, s);
    check_device_error(c, s);
  }
  if (schur) {
    // the root front holds exactly the GenEO columns, in order, at the top level
    const int r = nf - 1;
    const int64_t nh = schur->nh;
    if (F[r].npiv != nh || F[r].level != nlev - 1 || !F[r].upd.empty())
      throw Error(GENEO_ERR_CUDA, "internal: GenEO root front");
    check_device_error(c, s);
    const int64_t ntr = fb.nt[r];
    std::vector<double> tiles((size_t)(ntr * (ntr + 1) / 2) * kTileElems);
    GENEO_CUDA(cudaMemcpyAsync(tiles.data(), M->L.p + fb.toff[r] * kTileElems,
                               sizeof(double) * tiles.size(), cudaMemcpyDeviceToHost, s));
    GENEO_CUDA(cudaStreamSynchronize(s));
    schur->S.assign((size_t)(nh * nh), 0.0);
    for (int64_t i = 0; i < nh; ++i)
      for (int64_t j = 0; j <= i; ++j) {
        const int64_t I = i / kTile, J = j / kTile;
        const double v =
            tiles[(size_t)((I * (I + 1) / 2 + J) * kTileElems + (i % kTile) * kTile + j % kTile)];
        schur->S[i * nh + j] = schur->S[j * nh + i] = v;
      }
    c->mf.reset();
    return;
  }
  // --- inverses of the pivot blocks
  M->Y.alloc(tile_elems(fb));
  int maxpt = 0;
  for (int f = 0; f < nf; ++f) maxpt = std::max(maxpt, h_npivt[f]);
  pivot_block_inverse(fb, M->L.p, M->Y.p, M->dinv.p, M->dtoff.p, M->npivt.p, maxpt, s);
  check_device_error(c, s);
  mf_reserve(c, 1);
  M->factor_bytes = M->L.bytes() + M->Y.bytes();
  GENEO_CUDA(cudaStreamSynchronize(s));
}

// solve buffers for k right-hand-side columns
void mf_reserve(geneo_ctx *c, int k) {
  Multifrontal &M = *c->mf;
  if (k <= M.kcap) return;
  cudaStream_t s = c->stream;
  const int64_t vlen = M.fb.vlen, n0 = c->n0;
  M.wbuf.alloc(vlen * k);
  M.ybuf.alloc(vlen * k);
  M.tbuf.alloc(vlen * k);
  M.wbuf.zero(s);
  M.ybuf.zero(s);
  M.tbuf.zero(s);
  M.cpos.alloc(n0 * k);
  M.xpos.alloc(n0 * k);
  M.part.alloc((int64_t)M.nslot * kTile * k);
  M.cnt.alloc((int64_t)M.ncnt * k);
  M.cnt.zero(s);
  GENEO_CUDA(cudaStreamSynchronize(s));
  M.kcap = k;
}

int64_t mf_factor_bytes(const geneo_ctx *c) { return c->mf ? c->mf->factor_bytes : 0; }
int64_t mf_solve_bytes(const geneo_ctx *c) {
  return c->mf ? c->mf->solve_tiles * (int64_t)kTileElems * (int64_t)sizeof(double) : 0;
}

// y (column order, n0 per column, k columns) = E^-1 t
void mf_solve(geneo_ctx *c, const double *t, double *y, cudaStream_t s, int k) {
  Multifrontal &M = *c->mf;
  TileBatch &fb = M.fb;
  const int64_t n0 = c->n0;
  if (k > M.kcap) throw Error(GENEO_ERR_STATE, "internal: coarse solve buffers too small");
  k_perm<<<dim3(grid_for(n0, 256), k), 256, 0, s>>>(M.pos.p, t, M.cpos.p, n0, 1);
  MfArgs al{M.npivt.p, M.npiv.p, M.npivp.p, M.nupd.p, M.first.p, M.uoff.p, M.upos.p,
            fb.d_toff.p, fb.d_voff.p, M.L.p, M.wbuf.p, M.ybuf.p, M.tbuf.p, M.xpos.p,
            M.part.p, M.cnt.p, k, fb.vlen, n0, (int64_t)M.nslot * kTile, M.ncnt};
  MfArgs ay = al;
  ay.T = M.Y.p;
  const int nlev = (int)M.levels.size();
  for (int lv = 0; lv < nlev; ++lv) {
    MfLevel &Lv = M.levels[lv];
    k_mf_gather<<<dim3(grid_for(Lv.nrows, 256), k), 256, 0, s>>>(
        Lv.rf.p, Lv.rl.p, Lv.gptr.p, Lv.gidx.p, M.first.p, M.npiv.p, fb.d_voff.p, Lv.nrows, n0,
        fb.vlen, M.cpos.p, M.wbuf.p);
    if (Lv.ntask[0]) k_mf_tiles<0><<<Lv.ntask[0] * k, 256, 0, s>>>(Lv.task[0].p, ay);
    if (Lv.ntask[1]) k_mf_tiles<1><<<Lv.ntask[1] * k, 256, 0, s>>>(Lv.task[1].p, al);
  }
  for (int lv = nlev - 1; lv >= 0; --lv) {
    MfLevel &Lv = M.levels[lv];
    if (Lv.ntask[2]) k_mf_tiles<2><<<Lv.ntask[2] * k, 256, 0, s>>>(Lv.task[2].p, al);
    if (Lv.ntask[3]) k_mf_tiles<3><<<Lv.ntask[3] * k, 256, 0, s>>>(Lv.task[3].p, ay);
  }
  k_perm<<<dim3(grid_for(n0, 256), k), 256, 0, s>>>(M.pos.p, M.xpos.p, y, n0, 0);
  GENEO_CHECK_LAUNCH();
}

int mf_launches_per_solve(const geneo_ctx *c) {
  int n = 2;
  for (const MfLevel &Lv : c->mf->levels)
    n += 1 + (Lv.ntask[0] > 0) + (Lv.ntask[1] > 0) + (Lv.ntask[2] > 0) + (Lv.ntask[3] > 0);
  return n;
}

}  // namespace geneo
