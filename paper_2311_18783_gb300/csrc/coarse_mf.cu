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

#include "bulk.cuh"
#include "setup.hpp"

namespace geneo {

namespace {
constexpr int kLeafDefault = 256;
constexpr int kChunk = 4;     // tiles per task of the solve's tile GEMVs
constexpr int kColGroup = 4;  // right-hand-side columns one CTA applies a task's tiles to

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

// Shared memory of one tile task.
struct MfShared {
  double red[8][kTile];
  double vec[kTile];
  double xs[kChunk * kTile];
  int last;
};

// Offset (in tiles, from the factor's base) of tile q of a task.
template <int kMode>
__device__ __forceinline__ int64_t mf_tile_index(const MfTask &tk, const MfArgs &a, int q) {
  const int O = tk.I, K = tk.j0 + q;
  return kMode <= 1 ? a.toff[tk.f] + (int64_t)O * (O + 1) / 2 + K
                    : a.toff[tk.f] + (int64_t)K * (K + 1) / 2 + O;
}

// Factor tiles of a task into registers (warp w rows 8w..8w+7, lane l
// columns 2l, 2l+1), all issued before any use so their DRAM latencies
// overlap.  Reads only the factor and the front offsets, which no solve
// writes.
template <int kMode>
__device__ __forceinline__ void mf_load(const MfTask &tk, const MfArgs &a, const double *T,
                                        double2 (&v)[kChunk][8]) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int nk = tk.j1 - tk.j0;  // tiles of this task, at most kChunk
#pragma unroll
  for (int q = 0; q < kChunk; ++q) {
    if (q < nk) {
      const double *t = T + mf_tile_index<kMode>(tk, a, q) * kTileElems;
#pragma unroll
      for (int r = 0; r < 8; ++r)
        v[q][r] = __ldg(reinterpret_cast<const double2 *>(t + (w * 8 + r) * kTile + 2 * l));
    }
  }
}

// The rest of a task for right-hand side `col`: input entries, the tile
// GEMV, the split-K reduction and the output.  tile(q, r) gives the two
// entries (row 8w + r, columns 2l, 2l + 1) of the task's tile q that thread
// (warp w, lane l) multiplies.
template <int kMode, class TileAt>
__device__ __forceinline__ void mf_finish(const MfTask &tk, MfArgs a, int64_t col, TileAt tile,
                                          MfShared &sh) {
  a.wbuf += col * a.ldv;
  a.ybuf += col * a.ldv;
  a.tbuf += col * a.ldv;
  a.xpos += col * a.ldx;
  a.part += col * a.ldp;
  a.cnt += col * a.ldc;
  const int f = tk.f, O = tk.I;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int64_t vo = a.voff[f];
  const int nk = tk.j1 - tk.j0;
  if (kMode <= 1) {
    // row modes: y_O = sum_K T(O, K) x_K
    const double *vin = kMode == 0 ? a.wbuf : a.ybuf;
    double2 x[kChunk];
#pragma unroll
    for (int q = 0; q < kChunk; ++q)
      if (q < nk)
        x[q] = __ldcg(reinterpret_cast<const double2 *>(vin + vo + (int64_t)(tk.j0 + q) * kTile + 2 * l));
    double acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = 0.0;
#pragma unroll
    for (int q = 0; q < kChunk; ++q)
      if (q < nk)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const double2 t = tile(q, r);
          acc[r] = fma(t.x, x[q].x, fma(t.y, x[q].y, acc[r]));
        }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      double vv = acc[r];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) vv += __shfl_xor_sync(0xffffffffu, vv, o);
      if (l == 0) sh.vec[w * 8 + r] = vv;
    }
  } else {
    // column modes: y_O = sum_K T(K, O)^T x_K.  The input entries of the
    // task's rows are staged in shared memory first (phase 2 gathers them
    // through the update-row map, all in parallel)
    for (int e = threadIdx.x; e < nk * kTile; e += blockDim.x) {
      const int64_t row = (int64_t)tk.j0 * kTile + e;
      double xv;
      if (kMode == 2) {
        const int64_t u = row - a.npivp[f];
        xv = (u >= 0 && u < a.nupd[f]) ? __ldcg(a.xpos + a.upos[a.uoff[f] + u]) : 0.0;
      } else {
        xv = __ldcg(a.tbuf + vo + row);
      }
      sh.xs[e] = xv;
    }
    __syncthreads();
    double c0 = 0.0, c1 = 0.0;
#pragma unroll
    for (int q = 0; q < kChunk; ++q)
      if (q < nk)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const double xv = sh.xs[q * kTile + w * 8 + r];
          const double2 t = tile(q, r);
          c0 = fma(t.x, xv, c0);
          c1 = fma(t.y, xv, c1);
        }
    sh.red[w][2 * l] = c0;
    sh.red[w][2 * l + 1] = c1;
    __syncthreads();
    if (threadIdx.x < kTile) {
      double vv = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) vv += sh.red[q][threadIdx.x];
      sh.vec[threadIdx.x] = vv;
    }
  }
  __syncthreads();
  if (tk.nch > 1) {
    if (threadIdx.x < kTile) {
      a.part[(int64_t)tk.slot * kTile + threadIdx.x] = sh.vec[threadIdx.x];
      __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      sh.last = atomicAdd(&a.cnt[tk.cnt], 1) == tk.nch - 1;
    }
    __syncthreads();
    if (!sh.last) return;
    __threadfence();
    if (threadIdx.x < kTile) {
      double v = 0.0;
      for (int k = 0; k < tk.nch; ++k) v += __ldcg(a.part + (int64_t)(tk.rbase + k) * kTile + threadIdx.x);
      sh.vec[threadIdx.x] = v;
    }
    if (threadIdx.x == 0) a.cnt[tk.cnt] = 0;
    __syncthreads();
  }
  if (threadIdx.x < kTile) {
    const int64_t idx = (int64_t)O * kTile + threadIdx.x;
    const double v = sh.vec[threadIdx.x];
    if (kMode == 0) a.ybuf[vo + idx] = v;
    else if (kMode == 1) a.wbuf[vo + idx] = __ldcg(a.wbuf + vo + idx) - v;
    else if (kMode == 2) a.tbuf[vo + idx] = __ldcg(a.ybuf + vo + idx) - v;
    else if (idx < a.npiv[f]) a.xpos[a.first[f] + idx] = v;
  }
}

// One launch per (level, phase): blockIdx.x = task * ng + g.  CTA g of a
// task loads the task's tiles into registers once and applies them to the
// right-hand-side columns g kColGroup .. (g + 1) kColGroup - 1, one after
// another (ng = ceil(k / kColGroup) groups; one column per CTA when k = 1)
template <int kMode>
__global__ void __launch_bounds__(256) k_mf_tiles(const MfTask *__restrict__ tasks, MfArgs a,
                                                  int ng) {
  __shared__ MfShared sh;
  const int ti = blockIdx.x / ng, g = blockIdx.x - ti * ng;
  const MfTask tk = tasks[ti];
  double2 v[kChunk][8];
  mf_load<kMode>(tk, a, a.T, v);
  const int c1 = min(a.k, (g + 1) * kColGroup);
  for (int col = g * kColGroup; col < c1; ++col) {
    mf_finish<kMode>(tk, a, col, [&](int q, int r) { return v[q][r]; }, sh);
    __syncthreads();  // shared memory is reused by the next column
  }
}

// ---- the whole solve in one cooperative launch
//
// The steps of the level-by-level solve (permutation in, per level the
// gather and phases 0 and 1, per level downwards phases 2 and 3,
// permutation out) run in order, separated by a grid-wide barrier; the CTAs
// (all resident) stride over each step's items.  The factor tiles of a CTA's
// items stream through a ring of shared-memory slots filled by bulk copies
// ahead of use, across steps and barriers (the factor does not change during
// a solve), so tile latencies overlap the compute, the reductions and the
// barriers.  Every item computes
// exactly what its launch of the level-by-level path computes, in the same
// order, so both paths give identical results.  Vectors that a step
// writes are read through L2 (ld.global.cg): a CTA's L1 may still hold a
// line that another CTA has rewritten since (fronts adjacent in the
// elimination order share lines of the solution vector).

enum MfStepKind : int32_t { kStepPermIn = 0, kStepGather = 1, kStepTiles = 2, kStepPermOut = 6 };

struct MfStep {
  int32_t kind;  // MfStepKind; kStepTiles + p for tile phase p
  int32_t ntask;
  const MfTask *tasks;
  const int32_t *rf, *rl;
  const int64_t *gptr, *gidx;
  int64_t nrows;
};

struct MfPersistArgs {
  const MfStep *steps;
  int nsteps;
  MfArgs a;  // a.T unused: TL (phases 1, 2) and TY (phases 0, 3)
  const double *TL, *TY;
  const int64_t *pos, *first, *voff;
  const int32_t *npiv;
  const double *t;  // right-hand sides, column order, n0 each
  double *y;        // solutions, column order
  double *cpos;
  int64_t n0, vlen;
  unsigned *bar;    // [0] arrivals, [1] generation; zeroed before every launch
  int *err;
  long long *stamps;  // null, or clock64 of CTA 0 at every step start and at its end
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier (sense by generation count).  The generation is read
// before arriving; it can only move once every CTA, this one included, has
// arrived.  Thread 0 polls for about two seconds at most; past that the
// kernel records kDevTimeout and every CTA leaves (false).
__device__ __forceinline__ bool mf_grid_barrier(unsigned *bar, int *err, int &ok_sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g = ld_acquire_u32(bar + 1);
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (ld_acquire_u32(bar + 1) == g) {
        if (clock64() - t0 > 4000000000LL) {
          atomicCAS(err, kDevOk, kDevTimeout);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

// Shared memory of the single-launch solve beyond MfShared: a ring of
// kRing factor tiles and their mbarriers.
constexpr int kRing = 6;
constexpr size_t kMfPersistSmem = (size_t)kRing * kTileElems * sizeof(double) + kRing * 8;

__device__ __forceinline__ void mf_stamp(const MfPersistArgs &p, int st) {
  if (p.stamps && blockIdx.x == 0 && threadIdx.x == 0) p.stamps[st] = clock64();
}

// Offset (in tiles) of tile q of a task in tile phase `mode` (runtime form
// of mf_tile_index).
__device__ __forceinline__ int64_t mf_tile_at(const MfTask &tk, const int64_t *toff, int mode,
                                              int q) {
  const int O = tk.I, K = tk.j0 + q;
  return mode <= 1 ? toff[tk.f] + (int64_t)O * (O + 1) / 2 + K
                   : toff[tk.f] + (int64_t)K * (K + 1) / 2 + O;
}

// The tile stream of one CTA: the tiles of its items (it = blockIdx.x +
// j gridDim.x of every tile step), in the order it consumes them.  Thread 0
// issues them into the ring ahead of use, across steps and barriers: the
// factor does not change during a solve.
struct MfProducer {
  int st, it, q, nk, mode, nitems;
  MfTask tk;
  const MfTask *tasks;
  long long issued;

  // move to the next tile of the stream from (st, it, q); false at its end
  __device__ bool settle(const MfPersistArgs &p) {
    const int k = p.a.k;
    while (st < p.nsteps) {
      if (nitems > 0 && it < nitems) {
        if (q == 0 || nk < 0) {
          tk = tasks[it / k];
          nk = tk.j1 - tk.j0;
        }
        if (q < nk) return true;
        it += gridDim.x;
        q = 0;
        nk = -1;
        continue;
      }
      ++st;
      it = blockIdx.x;
      q = 0;
      nk = -1;
      nitems = 0;
      if (st < p.nsteps) {
        const MfStep S = p.steps[st];
        if (S.kind >= kStepTiles && S.kind < kStepPermOut) {
          mode = S.kind - kStepTiles;
          nitems = S.ntask * k;
          tasks = S.tasks;
        }
      }
    }
    return false;
  }

  // issue tiles while the ring has room (thread 0)
  __device__ void fill(const MfPersistArgs &p, long long consumed, double *ring, uint64_t *bars) {
    while (issued - consumed < kRing && settle(p)) {
      const int slot = (int)(issued % kRing);
      const double *T = (mode == 0 || mode == 3) ? p.TY : p.TL;
      fence_proxy_async();  // generic-proxy reads of the slot's last tile come first
      mbar_expect_tx(&bars[slot], (uint32_t)(kTileElems * sizeof(double)));
      bulk_g2s(ring + (size_t)slot * kTileElems, T + mf_tile_at(tk, p.a.toff, mode, q) * kTileElems,
               (uint32_t)(kTileElems * sizeof(double)), &bars[slot]);
      ++issued;
      ++q;
    }
  }
};

template <int kMode>
__device__ __forceinline__ bool mf_tile_step(const MfStep &S, int st, const MfPersistArgs &p,
                                             bool sync, double *ring, uint64_t *bars,
                                             MfProducer &pr, long long &consumed, MfShared &sh,
                                             int &ok_sh) {
  const int k = p.a.k;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int nitems = S.ntask * k;  // at most 2^31 (tasks x 16 columns)
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int ti = it / k, col = it - ti * k;
    const MfTask tk = S.tasks[ti];
    const int nk = tk.j1 - tk.j0;
    if (threadIdx.x == 0) pr.fill(p, consumed, ring, bars);
    if (sync) {
      if (!mf_grid_barrier(p.bar, p.err, ok_sh)) return false;
      sync = false;
      mf_stamp(p, st);
    }
    bool ok = true;
    for (int q = 0; q < nk; ++q) {
      const long long u = consumed + q;
      ok = ok && mbar_wait_bounded(&bars[(int)(u % kRing)], (uint32_t)((u / kRing) & 1));
    }
    // every thread of the CTA takes the same decision
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) atomicCAS(p.err, kDevOk, kDevTimeout);
      return false;
    }
    const long long c0 = consumed;
    mf_finish<kMode>(tk, p.a, col,
                     [&](int q, int r) {
                       return *reinterpret_cast<const double2 *>(
                           ring + (size_t)((c0 + q) % kRing) * kTileElems + (w * 8 + r) * kTile +
                           2 * l);
                     },
                     sh);
    __syncthreads();  // the item's slots are free again
    consumed += nk;
  }
  if (sync) {
    if (threadIdx.x == 0) pr.fill(p, consumed, ring, bars);
    if (!mf_grid_barrier(p.bar, p.err, ok_sh)) return false;
    mf_stamp(p, st);
  }
  return true;
}

__global__ void __launch_bounds__(256, 1) k_mf_solve_persistent(MfPersistArgs p) {
  __shared__ MfShared sh;
  __shared__ int ok_sh;
  extern __shared__ __align__(128) unsigned char mf_dyn[];
  double *ring = reinterpret_cast<double *>(mf_dyn);
  uint64_t *bars = reinterpret_cast<uint64_t *>(mf_dyn + (size_t)kRing * kTileElems * sizeof(double));
  if (threadIdx.x == 0) {
    for (int i = 0; i < kRing; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
  }
  __syncthreads();
  MfProducer pr;
  pr.st = -1;
  pr.it = 0;
  pr.q = 0;
  pr.nk = -1;
  pr.mode = 0;
  pr.nitems = 0;
  pr.tasks = nullptr;
  pr.issued = 0;
  long long consumed = 0;
  const int k = p.a.k;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool ok = true;
  mf_stamp(p, 0);
  for (int st = 0; st < p.nsteps && ok; ++st) {
    const MfStep S = p.steps[st];
    const bool sync = st > 0;
    if (S.kind >= kStepTiles && S.kind < kStepPermOut) {
      switch (S.kind - kStepTiles) {
        case 0: ok = mf_tile_step<0>(S, st, p, sync, ring, bars, pr, consumed, sh, ok_sh); break;
        case 1: ok = mf_tile_step<1>(S, st, p, sync, ring, bars, pr, consumed, sh, ok_sh); break;
        case 2: ok = mf_tile_step<2>(S, st, p, sync, ring, bars, pr, consumed, sh, ok_sh); break;
        default: ok = mf_tile_step<3>(S, st, p, sync, ring, bars, pr, consumed, sh, ok_sh); break;
      }
      continue;
    }
    if (threadIdx.x == 0) pr.fill(p, consumed, ring, bars);
    if (sync) {
      if (!mf_grid_barrier(p.bar, p.err, ok_sh)) {
        ok = false;
        break;
      }
      mf_stamp(p, st);
    }
    if (S.kind == kStepPermIn || S.kind == kStepPermOut) {
      for (int col = 0; col < k; ++col) {
        const int64_t co = (int64_t)col * p.n0;
        for (int64_t i = gtid; i < p.n0; i += gthreads) {
          if (S.kind == kStepPermIn) p.cpos[co + p.pos[i]] = p.t[co + i];
          else p.y[co + i] = __ldcg(p.a.xpos + co + p.pos[i]);
        }
      }
    } else {
      // forward gather (k_mf_gather)
      for (int col = 0; col < k; ++col) {
        const double *cp = p.cpos + (int64_t)col * p.n0;
        double *w = p.a.wbuf + (int64_t)col * p.vlen;
        for (int64_t r = gtid; r < S.nrows; r += gthreads) {
          const int f = S.rf[r], l = S.rl[r];
          double v = l < p.npiv[f] ? __ldcg(cp + p.first[f] + l) : 0.0;
          for (int64_t e = S.gptr[r]; e < S.gptr[r + 1]; ++e) v += __ldcg(w + S.gidx[e]);
          w[p.voff[f] + l] = v;
        }
      }
    }
  }
  if (ok) mf_stamp(p, p.nsteps);
  // copies still in flight (a failed wait, or none) land before the CTA leaves
  if (threadIdx.x == 0)
    for (long long u = consumed; u < pr.issued; ++u)
      mbar_wait_bounded(&bars[(int)(u % kRing)], (uint32_t)((u / kRing) & 1));
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
  int64_t ntiles[4] = {0, 0, 0, 0};                 // factor tiles each phase reads
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
  // the single-launch solve: its steps, barrier words and grid (0 CTAs:
  // cooperative launches unavailable)
  DevBuf<MfStep> steps;
  int nsteps = 0;
  DevBuf<unsigned> bar;
  int persist_ctas = 0;
  // per step: kind, level, items, factor bytes; and the SM clock of CTA 0
  // at the start of every step of the last profiled solve
  std::vector<double> step_info;
  DevBuf<long long> stamps;
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
        Lv.ntiles[ph] += std::max(0, o1 - o0);
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
  // steps of the single-launch solve, in the order of the level-by-level one
  {
    std::vector<MfStep> st;
    std::vector<double> &info = M->step_info;
    auto note = [&](int kind, int lv, int64_t items, int64_t tiles) {
      info.insert(info.end(), {(double)kind, (double)lv, (double)items,
                               (double)tiles * kTileElems * sizeof(double)});
    };
    MfStep e{};
    e.kind = kStepPermIn;
    st.push_back(e);
    note(kStepPermIn, -1, n0, 0);
    for (int lv = 0; lv < nlev; ++lv) {
      const MfLevel &Lv = M->levels[lv];
      MfStep g{};
      g.kind = kStepGather;
      g.rf = Lv.rf.p;
      g.rl = Lv.rl.p;
      g.gptr = Lv.gptr.p;
      g.gidx = Lv.gidx.p;
      g.nrows = Lv.nrows;
      if (Lv.nrows > 0) {
        st.push_back(g);
        note(kStepGather, lv, Lv.nrows, 0);
      }
      for (int ph = 0; ph < 2; ++ph)
        if (Lv.ntask[ph]) {
          MfStep t{};
          t.kind = kStepTiles + ph;
          t.ntask = Lv.ntask[ph];
          t.tasks = Lv.task[ph].p;
          st.push_back(t);
          note(t.kind, lv, Lv.ntask[ph], Lv.ntiles[ph]);
        }
    }
    for (int lv = nlev - 1; lv >= 0; --lv) {
      const MfLevel &Lv = M->levels[lv];
      for (int ph = 2; ph < 4; ++ph)
        if (Lv.ntask[ph]) {
          MfStep t{};
          t.kind = kStepTiles + ph;
          t.ntask = Lv.ntask[ph];
          t.tasks = Lv.task[ph].p;
          st.push_back(t);
          note(t.kind, lv, Lv.ntask[ph], Lv.ntiles[ph]);
        }
    }
    e.kind = kStepPermOut;
    st.push_back(e);
    note(kStepPermOut, -1, n0, 0);
    M->stamps.alloc((int64_t)st.size() + 1);
    M->stamps.zero(s);
    M->steps.upload(st, s);
    M->nsteps = (int)st.size();
    M->bar.alloc(2);
    M->bar.zero(s);
    int dev = 0, coop = 0, nsm = 0, per_sm = 0;
    GENEO_CUDA(cudaGetDevice(&dev));
    GENEO_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    GENEO_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    GENEO_CUDA(cudaFuncSetAttribute(k_mf_solve_persistent,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kMfPersistSmem));
    GENEO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mf_solve_persistent, 256,
                                                             kMfPersistSmem));
    M->persist_ctas = coop ? nsm * std::min(per_sm, 2) : 0;
  }
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
  MfArgs al{M.npivt.p, M.npiv.p, M.npivp.p, M.nupd.p, M.first.p, M.uoff.p, M.upos.p,
            fb.d_toff.p, fb.d_voff.p, M.L.p, M.wbuf.p, M.ybuf.p, M.tbuf.p, M.xpos.p,
            M.part.p, M.cnt.p, k, fb.vlen, n0, (int64_t)M.nslot * kTile, M.ncnt};
  MfArgs ay = al;
  ay.T = M.Y.p;
  if (c->mf_persist && M.persist_ctas > 0) {
    MfPersistArgs pa{M.steps.p, M.nsteps, al, M.L.p, M.Y.p, M.pos.p, M.first.p, fb.d_voff.p,
                     M.npiv.p, t, y, M.cpos.p, n0, fb.vlen, M.bar.p, c->d_err.p,
                     c->prof ? M.stamps.p : nullptr};
    // barrier words start from zero on every launch, also after a launch
    // that gave up at a barrier
    GENEO_CUDA(cudaMemsetAsync(M.bar.p, 0, 2 * sizeof(unsigned), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)M.persist_ctas);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = kMfPersistSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    GENEO_CUDA(cudaLaunchKernelEx(&cfg, k_mf_solve_persistent, pa));
    return;
  }
  k_perm<<<dim3(grid_for(n0, 256), k), 256, 0, s>>>(M.pos.p, t, M.cpos.p, n0, 1);
  const int nlev = (int)M.levels.size();
  const int ng = (k + kColGroup - 1) / kColGroup;
  for (int lv = 0; lv < nlev; ++lv) {
    MfLevel &Lv = M.levels[lv];
    k_mf_gather<<<dim3(grid_for(Lv.nrows, 256), k), 256, 0, s>>>(
        Lv.rf.p, Lv.rl.p, Lv.gptr.p, Lv.gidx.p, M.first.p, M.npiv.p, fb.d_voff.p, Lv.nrows, n0,
        fb.vlen, M.cpos.p, M.wbuf.p);
    if (Lv.ntask[0]) k_mf_tiles<0><<<Lv.ntask[0] * ng, 256, 0, s>>>(Lv.task[0].p, ay, ng);
    if (Lv.ntask[1]) k_mf_tiles<1><<<Lv.ntask[1] * ng, 256, 0, s>>>(Lv.task[1].p, al, ng);
  }
  for (int lv = nlev - 1; lv >= 0; --lv) {
    MfLevel &Lv = M.levels[lv];
    if (Lv.ntask[2]) k_mf_tiles<2><<<Lv.ntask[2] * ng, 256, 0, s>>>(Lv.task[2].p, al, ng);
    if (Lv.ntask[3]) k_mf_tiles<3><<<Lv.ntask[3] * ng, 256, 0, s>>>(Lv.task[3].p, ay, ng);
  }
  k_perm<<<dim3(grid_for(n0, 256), k), 256, 0, s>>>(M.pos.p, M.xpos.p, y, n0, 0);
  GENEO_CHECK_LAUNCH();
}

bool mf_single_launch_available(const geneo_ctx *c) {
  return c->mf && c->mf->persist_ctas > 0;
}

std::vector<double> mf_step_profile(const geneo_ctx *c) {
  std::vector<double> out;
  if (!c->mf) return out;
  const Multifrontal &M = *c->mf;
  const std::vector<long long> t = M.stamps.download(c->stream);
  for (int i = 0; i < M.nsteps; ++i) {
    out.insert(out.end(), M.step_info.begin() + 4 * i, M.step_info.begin() + 4 * i + 4);
    out.push_back((double)(t[i + 1] - t[i]));
  }
  return out;
}

int mf_launches_per_solve(const geneo_ctx *c) {
  if (c->mf_persist && c->mf->persist_ctas > 0) return 1;
  int n = 2;
  for (const MfLevel &Lv : c->mf->levels)
    n += 1 + (Lv.ntask[0] > 0) + (Lv.ntask[1] > 0) + (Lv.ntask[2] > 0) + (Lv.ntask[3] > 0);
  return n;
}

}  // namespace geneo
