// Batched tile-packed symmetric matrices: explicit inversion by tiled
// Cholesky (float64) and a streaming SYMV whose 64x64 tiles are staged in
// shared memory by cp.async.bulk copies completed on mbarriers.
//
// The local solves A_i^-1 of Sec. 2, eq. "AS", are applied as explicit
// inverses: every tile is read once per application and the work of all
// subdomains is spread over all SMs.
#include "dense.cuh"
#include "bulk.cuh"

#include <algorithm>
#include <cmath>
#include <queue>

namespace geneo {

int device_sm_count() {
  int dev = 0, n = 0;
  GENEO_CUDA(cudaGetDevice(&dev));
  GENEO_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  return n;
}

void TileBatch::layout(const std::vector<int64_t> &dims) {
  nmat = (int)dims.size();
  dim = dims;
  nt.resize(nmat);
  toff.resize(nmat + 1);
  voff.resize(nmat + 1);
  toff[0] = voff[0] = 0;
  maxnt = 0;
  for (int m = 0; m < nmat; ++m) {
    nt[m] = (int32_t)((dims[m] + kTile - 1) / kTile);
    maxnt = std::max(maxnt, nt[m]);
    toff[m + 1] = toff[m] + (int64_t)nt[m] * (nt[m] + 1) / 2;
    voff[m + 1] = voff[m] + (int64_t)nt[m] * kTile;
  }
  ntiles = toff[nmat];
  vlen = voff[nmat];
}

void TileBatch::upload_meta(cudaStream_t s) {
  d_nt.upload(nt, s);
  d_toff.upload(toff, s);
  d_voff.upload(voff, s);
  std::vector<int32_t> vm, vi;
  for (int m = 0; m < nmat; ++m)
    for (int I = 0; I < nt[m]; ++I) {
      vm.push_back(m);
      vi.push_back(I);
    }
  d_vrow_m.upload(vm, s);
  d_vrow_I.upload(vi, s);
  rowpart.alloc(vlen);
  colpart.alloc(ntiles * (int64_t)kTile);
}

// Longest-processing-time assignment of tile rows (strips) to persistent CTAs.
void TileBatch::schedule(int nctas, cudaStream_t s) {
  struct Strip { int32_t m, I; };
  std::vector<Strip> strips;
  for (int m = 0; m < nmat; ++m)
    for (int I = 0; I < nt[m]; ++I) strips.push_back({m, I});
  std::stable_sort(strips.begin(), strips.end(),
                   [](const Strip &a, const Strip &b) { return a.I > b.I; });
  nctas = std::max(1, std::min<int>(nctas, (int)strips.size()));
  using Load = std::pair<int64_t, int>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
  for (int c = 0; c < nctas; ++c) pq.push({0, c});
  std::vector<std::vector<Strip>> per(nctas);
  for (const Strip &st : strips) {
    Load l = pq.top();
    pq.pop();
    per[l.second].push_back(st);
    pq.push({l.first + st.I + 1, l.second});
  }
  std::vector<int32_t> sm, si, off(1, 0);
  for (int c = 0; c < nctas; ++c) {
    for (const Strip &st : per[c]) {
      sm.push_back(st.m);
      si.push_back(st.I);
    }
    off.push_back((int32_t)sm.size());
  }
  sched_ctas = nctas;
  d_strip_m.upload(sm, s);
  d_strip_I.upload(si, s);
  d_cta_off.upload(off, s);
  base_ctas = nctas;
  for (auto &e : extra) e.nctas = 0;  // rebuilt on demand
}

// Schedule with cps persistent CTAs per SM of the base schedule (cps = 1 is
// the base schedule itself); built once per cps.
const TileBatch::Sched &TileBatch::sched_for(int cps) {
  if (cps <= 1) {
    base.nctas = sched_ctas;
    base.strip_m.p = d_strip_m.p;
    base.strip_I.p = d_strip_I.p;
    base.cta_off.p = d_cta_off.p;
    return base;
  }
  Sched &e = extra[std::min(cps, 4) - 2];
  if (e.nctas) return e;
  struct Strip { int32_t m, I; };
  std::vector<Strip> strips;
  for (int m = 0; m < nmat; ++m)
    for (int I = 0; I < nt[m]; ++I) strips.push_back({m, I});
  std::stable_sort(strips.begin(), strips.end(),
                   [](const Strip &a, const Strip &b) { return a.I > b.I; });
  const int nctas = std::max(1, std::min<int>(base_ctas * cps, (int)strips.size()));
  using Load = std::pair<int64_t, int>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
  for (int c = 0; c < nctas; ++c) pq.push({0, c});
  std::vector<std::vector<Strip>> per(nctas);
  for (const Strip &st : strips) {
    Load l = pq.top();
    pq.pop();
    per[l.second].push_back(st);
    pq.push({l.first + st.I + 1, l.second});
  }
  std::vector<int32_t> sm, si, off(1, 0);
  for (int c = 0; c < nctas; ++c) {
    for (const Strip &st : per[c]) {
      sm.push_back(st.m);
      si.push_back(st.I);
    }
    off.push_back((int32_t)sm.size());
  }
  e.own_m.upload(sm, 0);
  e.own_I.upload(si, 0);
  e.own_off.upload(off, 0);
  GENEO_CUDA(cudaStreamSynchronize(0));
  e.strip_m.p = e.own_m.p;
  e.strip_I.p = e.own_I.p;
  e.cta_off.p = e.own_off.p;
  e.nctas = nctas;
  return e;
}

// ---------------------------------------------------------------------------
// tile helpers


__device__ __forceinline__ int64_t tidx(int64_t toff, int I, int J) {
  return toff + (int64_t)I * (I + 1) / 2 + J;
}


// dst[r][c] = src[r][c] (transpose = false) or src[c][r] (transpose = true)
__device__ __forceinline__ void load_tile_smem(double *dst, const double *__restrict__ src,
                                               bool transpose) {
  for (int q = threadIdx.x; q < kTileElems; q += blockDim.x) {
    const int r = q >> 6, c = q & 63;
    const double v = src[q];
    if (transpose) dst[c * kLd + r] = v;
    else dst[r * kLd + c] = v;
  }
}


// ---------------------------------------------------------------------------
// Explicit SPD inverse by tiled Cholesky.  A = L L^T (POTRF on the diagonal
// tile, TRSM of the column panel with the inverted diagonal tile, SYRK/GEMM
// update of the trailing tiles); Y = L^-1 by tiled forward substitution on
// the identity; A^-1 = Y^T Y.  (A symmetric Gauss-Jordan sweep is not used:
// on matrices with the large gradient near-kernel of A_i = K_i + gamma M_i it
// loses several digits, while the Cholesky route keeps the forward error at
// kappa(A_i) u.)

// Unblocked Cholesky of the diagonal tile in shared memory, then the inverse
// of L_kk by 64 independent forward substitutions.  Writes L_kk (upper part
// zeroed) to the storage and L_kk^-1 to dinv.
__global__ void __launch_bounds__(256) k_potrf(double *data, const int32_t *nt,
                                               const int64_t *toff, const int64_t *dtoff,
                                               const int32_t *npiv, int k, double *dinv, int *err) {
  extern __shared__ double sh[];
  const int m = blockIdx.x;
  const int lim = npiv ? npiv[m] : nt[m];
  if (k >= lim) return;
  double *a = sh, *x = sh + kTile * kLd;
  double *tile = data + tidx(toff[m], k, k) * kTileElems;
  load_tile_smem(a, tile, false);
  __syncthreads();
  for (int p = 0; p < kTile; ++p) {
    double d = a[p * kLd + p];
    if (!(d > 0.0) || !isfinite(d)) {
      if (threadIdx.x == 0) atomicCAS(err, kDevOk, kDevNotSPD);
      d = 1.0;
    }
    d = sqrt(d);
    __syncthreads();
    if (threadIdx.x < kTile) {
      const int r = threadIdx.x;
      if (r > p) a[r * kLd + p] /= d;
      else if (r == p) a[p * kLd + p] = d;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kTileElems; q += blockDim.x) {
      const int r = q >> 6, c = q & 63;
      if (c > p && r >= c) a[r * kLd + c] -= a[r * kLd + p] * a[c * kLd + p];
    }
    __syncthreads();
  }
  // X = L^-1: thread c solves L x = e_c (x[r] = 0 for r < c)
  if (threadIdx.x < kTile) {
    const int c = threadIdx.x;
    for (int r = 0; r < kTile; ++r) {
      double v = (r == c) ? 1.0 : 0.0;
      if (r >= c) {
        for (int t = c; t < r; ++t) v -= a[r * kLd + t] * x[t * kLd + c];
        v /= a[r * kLd + r];
      } else {
        v = 0.0;
      }
      x[r * kLd + c] = v;
    }
  }
  __syncthreads();
  double *Li = dinv + (dtoff[m] + k) * kTileElems;
  for (int q = threadIdx.x; q < kTileElems; q += blockDim.x) {
    const int r = q >> 6, c = q & 63;
    tile[q] = (c <= r) ? a[r * kLd + c] : 0.0;
    Li[q] = x[r * kLd + c];
  }
}

// L_Ik = A_Ik L_kk^-T for I > k
__global__ void __launch_bounds__(256) k_trsm(double *data, const int32_t *nt, const int64_t *toff,
                                              const int64_t *dtoff, const int32_t *npiv, int k,
                                              const double *dinv) {
  extern __shared__ double sh[];
  const int I = k + 1 + blockIdx.x, m = blockIdx.y;
  const int lim = npiv ? npiv[m] : nt[m];
  if (k >= lim || I >= nt[m]) return;
  double *As = sh, *Bs = sh + kTile * kLd;
  double *dst = data + tidx(toff[m], I, k) * kTileElems;
  load_tile_smem(As, dst, false);
  load_tile_smem(Bs, dinv + (dtoff[m] + k) * kTileElems, false);
  __syncthreads();
  double acc[4][4] = {};
  gemm_abt(As, Bs, acc);
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) dst[(4 * tr + i) * kTile + tc + 16 * j] = acc[i][j];
}

// A_IJ -= L_Ik L_Jk^T for k < J <= I (tiles enumerated from (k+1, k+1))
__global__ void __launch_bounds__(256) k_syrk(double *data, const int32_t *nt, const int64_t *toff,
                                              const int32_t *npiv, int k) {
  extern __shared__ double sh[];
  const int m = blockIdx.y;
  const int lim = npiv ? npiv[m] : nt[m];
  if (k >= lim) return;
  const int64_t rest = nt[m] - k - 1;
  const int64_t q = blockIdx.x;
  if (q >= rest * (rest + 1) / 2) return;
  int I, J;
  tile_I_J(q, I, J);
  I += k + 1;
  J += k + 1;
  double *As = sh, *Bs = sh + kTile * kLd;
  load_tile_smem(As, data + tidx(toff[m], I, k) * kTileElems, false);
  load_tile_smem(Bs, data + tidx(toff[m], J, k) * kTileElems, false);
  __syncthreads();
  double acc[4][4] = {};
  gemm_abt(As, Bs, acc);
  double *dst = data + tidx(toff[m], I, J) * kTileElems;
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) dst[(4 * tr + i) * kTile + tc + 16 * j] -= acc[i][j];
}

// forward substitution on the identity, step k:
//   Y_kj = L_kk^-1 B_kj  (j <= k), with B = I - (updates so far)
__global__ void __launch_bounds__(256) k_fwd_diag(double *Y, const int32_t *nt, const int64_t *toff,
                                                  const int64_t *dtoff, int k, const double *dinv,
                                                  const int32_t *lim) {
  extern __shared__ double sh[];
  const int j = blockIdx.x, m = blockIdx.y;
  if (k >= (lim ? lim[m] : nt[m]) || j > k) return;
  double *As = sh, *Bs = sh + kTile * kLd;
  double *dst = Y + tidx(toff[m], k, j) * kTileElems;
  load_tile_smem(As, dinv + (dtoff[m] + k) * kTileElems, false);
  load_tile_smem(Bs, dst, true);
  __syncthreads();
  double acc[4][4] = {};
  gemm_abt(As, Bs, acc);
  __syncthreads();
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) dst[(4 * tr + i) * kTile + tc + 16 * jj] = acc[i][jj];
}

//   B_Ij -= L_Ik Y_kj  (I > k, j <= k)
__global__ void __launch_bounds__(256) k_fwd_update(double *Y, const double *L, const int32_t *nt,
                                                    const int64_t *toff, int k, const int32_t *lim) {
  extern __shared__ double sh[];
  const int m = blockIdx.z;
  const int I = k + 1 + blockIdx.x, j = blockIdx.y;
  if (I >= (lim ? lim[m] : nt[m]) || j > k) return;
  double *As = sh, *Bs = sh + kTile * kLd;
  load_tile_smem(As, L + tidx(toff[m], I, k) * kTileElems, false);
  load_tile_smem(Bs, Y + tidx(toff[m], k, j) * kTileElems, true);
  __syncthreads();
  double acc[4][4] = {};
  gemm_abt(As, Bs, acc);
  double *dst = Y + tidx(toff[m], I, j) * kTileElems;
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) dst[(4 * tr + i) * kTile + tc + 16 * jj] -= acc[i][jj];
}

// X_IJ = sum_{K >= I} Y_KI^T Y_KJ (J <= I), written over the factor storage
__global__ void __launch_bounds__(256) k_lauum(double *X, const double *Y, const int32_t *nt,
                                               const int64_t *toff) {
  extern __shared__ double sh[];
  const int m = blockIdx.y;
  const int64_t ntm = nt[m];
  const int64_t q = blockIdx.x;
  if (q >= ntm * (ntm + 1) / 2) return;
  int I, J;
  tile_I_J(q, I, J);
  double *As = sh, *Bs = sh + kTile * kLd;
  double acc[4][4] = {};
  for (int K = I; K < ntm; ++K) {
    load_tile_smem(As, Y + tidx(toff[m], K, I) * kTileElems, true);
    load_tile_smem(Bs, Y + tidx(toff[m], K, J) * kTileElems, true);
    __syncthreads();
    gemm_abt(As, Bs, acc);
    __syncthreads();
  }
  double *dst = X + tidx(toff[m], I, J) * kTileElems;
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) dst[(4 * tr + i) * kTile + tc + 16 * j] = acc[i][j];
}

// symmetrise the diagonal tiles (X_II is computed in full)
__global__ void k_symmetrize_diag(double *X, const int32_t *nt, const int64_t *toff) {
  const int m = blockIdx.y, I = blockIdx.x;
  if (I >= nt[m]) return;
  double *t = X + tidx(toff[m], I, I) * kTileElems;
  for (int e = threadIdx.x; e < kTileElems; e += blockDim.x) {
    const int r = e >> 6, c = e & 63;
    if (r < c) {
      const double v = 0.5 * (t[r * kTile + c] + t[c * kTile + r]);
      t[r * kTile + c] = v;
      t[c * kTile + r] = v;
    }
  }
}

// B = identity in tile-packed storage
__global__ void k_identity(double *Y, const int32_t *nt, const int64_t *toff) {
  const int m = blockIdx.y, I = blockIdx.x;
  if (I >= nt[m]) return;
  double *t = Y + tidx(toff[m], I, I) * kTileElems;
  for (int r = threadIdx.x; r < kTile; r += blockDim.x) t[r * kTile + r] = 1.0;
}

__global__ void k_tiles_padding(double *data, const int32_t *nt, const int64_t *toff,
                                const int64_t *dim) {
  const int m = blockIdx.y;
  const int ntm = nt[m];
  const int64_t d = dim[m];
  for (int64_t r = d + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < (int64_t)ntm * kTile;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int I = (int)(r / kTile), rr = (int)(r % kTile);
    data[tidx(toff[m], I, I) * kTileElems + rr * kTile + rr] = 1.0;
  }
}

__global__ void k_cast_f32(const double *src, float *dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

int64_t spd_workspace_elems(const TileBatch &b) {
  int64_t diag = 0;
  for (int m = 0; m < b.nmat; ++m) diag += b.nt[m];
  return (b.ntiles + diag) * kTileElems;
}

static void set_smem_attrs() {
  static bool done = false;
  if (done) return;
  const int two = 2 * kTile * kLd * (int)sizeof(double);
  GENEO_CUDA(cudaFuncSetAttribute(k_potrf, cudaFuncAttributeMaxDynamicSharedMemorySize, two));
  GENEO_CUDA(cudaFuncSetAttribute(k_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, two));
  GENEO_CUDA(cudaFuncSetAttribute(k_syrk, cudaFuncAttributeMaxDynamicSharedMemorySize, two));
  GENEO_CUDA(cudaFuncSetAttribute(k_fwd_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, two));
  GENEO_CUDA(cudaFuncSetAttribute(k_fwd_update, cudaFuncAttributeMaxDynamicSharedMemorySize, two));
  GENEO_CUDA(cudaFuncSetAttribute(k_lauum, cudaFuncAttributeMaxDynamicSharedMemorySize, two));
  done = true;
}

void chol_factor(TileBatch &b, double *data, const int32_t *d_npiv, int nsteps, double *dinv,
                 const int64_t *d_dtoff, int *d_err, cudaStream_t s) {
  set_smem_attrs();
  const int two = 2 * kTile * kLd * (int)sizeof(double);
  for (int k = 0; k < nsteps; ++k) {
    k_potrf<<<b.nmat, 256, two, s>>>(data, b.d_nt.p, b.d_toff.p, d_dtoff, d_npiv, k, dinv, d_err);
    const int rest = b.maxnt - k - 1;
    if (rest > 0) {
      k_trsm<<<dim3(rest, b.nmat), 256, two, s>>>(data, b.d_nt.p, b.d_toff.p, d_dtoff, d_npiv, k,
                                                 dinv);
      const int64_t nq = (int64_t)rest * (rest + 1) / 2;
      k_syrk<<<dim3((unsigned)nq, b.nmat), 256, two, s>>>(data, b.d_nt.p, b.d_toff.p, d_npiv, k);
    }
  }
  GENEO_CHECK_LAUNCH();
}

void spd_invert(TileBatch &b, double *data, double *ws, int *d_err, cudaStream_t s) {
  set_smem_attrs();
  const int two = 2 * kTile * kLd * (int)sizeof(double);
  double *Y = ws;
  double *dinv = ws + b.ntiles * kTileElems;
  std::vector<int64_t> dtoff(b.nmat + 1, 0);
  for (int m = 0; m < b.nmat; ++m) dtoff[m + 1] = dtoff[m] + b.nt[m];
  DevBuf<int64_t> d_dtoff;
  d_dtoff.upload(dtoff, s);
  chol_factor(b, data, nullptr, b.maxnt, dinv, d_dtoff.p, d_err, s);
  GENEO_CUDA(cudaMemsetAsync(Y, 0, sizeof(double) * (size_t)tile_elems(b), s));
  k_identity<<<dim3(b.maxnt, b.nmat), 64, 0, s>>>(Y, b.d_nt.p, b.d_toff.p);
  for (int k = 0; k < b.maxnt; ++k) {
    k_fwd_diag<<<dim3(k + 1, b.nmat), 256, two, s>>>(Y, b.d_nt.p, b.d_toff.p, d_dtoff.p, k, dinv,
                                                     nullptr);
    const int rest = b.maxnt - k - 1;
    if (rest > 0)
      k_fwd_update<<<dim3(rest, k + 1, b.nmat), 256, two, s>>>(Y, data, b.d_nt.p, b.d_toff.p, k,
                                                               nullptr);
  }
  const int64_t maxT = (int64_t)b.maxnt * (b.maxnt + 1) / 2;
  k_lauum<<<dim3((unsigned)maxT, b.nmat), 256, two, s>>>(data, Y, b.d_nt.p, b.d_toff.p);
  k_symmetrize_diag<<<dim3(b.maxnt, b.nmat), 256, 0, s>>>(data, b.d_nt.p, b.d_toff.p);
  GENEO_CHECK_LAUNCH();
  GENEO_CUDA(cudaStreamSynchronize(s));
}

void pivot_block_inverse(TileBatch &b, const double *L, double *Y, const double *dinv,
                         const int64_t *d_dtoff, const int32_t *d_npiv, int max_npiv,
                         cudaStream_t s) {
  set_smem_attrs();
  const int two = 2 * kTile * kLd * (int)sizeof(double);
  GENEO_CUDA(cudaMemsetAsync(Y, 0, sizeof(double) * (size_t)tile_elems(b), s));
  k_identity<<<dim3(b.maxnt, b.nmat), 64, 0, s>>>(Y, b.d_nt.p, b.d_toff.p);
  for (int k = 0; k < max_npiv; ++k) {
    k_fwd_diag<<<dim3(k + 1, b.nmat), 256, two, s>>>(Y, b.d_nt.p, b.d_toff.p, d_dtoff, k, dinv,
                                                     d_npiv);
    const int rest = max_npiv - k - 1;
    if (rest > 0)
      k_fwd_update<<<dim3(rest, k + 1, b.nmat), 256, two, s>>>(Y, L, b.d_nt.p, b.d_toff.p, k,
                                                               d_npiv);
  }
  GENEO_CHECK_LAUNCH();
}

void tiles_init_padding(TileBatch &b, double *data, cudaStream_t s) {
  GENEO_CUDA(cudaMemsetAsync(data, 0, sizeof(double) * (size_t)tile_elems(b), s));
  DevBuf<int64_t> dd;
  dd.upload(b.dim, s);
  k_tiles_padding<<<dim3(1, b.nmat), 64, 0, s>>>(data, b.d_nt.p, b.d_toff.p, dd.p);
  GENEO_CHECK_LAUNCH();
  GENEO_CUDA(cudaStreamSynchronize(s));
}

void tiles_cast_f32(const TileBatch &b, const double *src, float *dst, cudaStream_t s) {
  const int64_t n = tile_elems(b);
  const unsigned g = std::min<int64_t>(grid_for(n, 256), 65535LL * 16);
  k_cast_f32<<<g, 256, 0, s>>>(src, dst, n);
  GENEO_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// Streaming SYMV.  Persistent CTAs walk their strips (tile rows) tile by tile;
// an elected thread keeps NST bulk copies in flight.  Each thread owns 8 rows
// x 2 columns of a tile: row partials accumulate over the strip, column
// partials (the mirrored upper triangle) are reduced across warps per tile.

template <typename T> struct Acc { using type = float; };
template <> struct Acc<double> { using type = double; };

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

// Tiles are consumed in batches of up to D tiles of one strip: one barrier
// after the D waits (also the uniform timeout decision), the D tiles'
// products, one barrier, then the column partials of the D tiles reduced
// across warps by all threads, and D new copies issued.  WARPS warps share a
// tile: each owns 64 / WARPS rows and lane l columns 2l, 2l + 1.
template <typename T, int NST, int D, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
    k_symv_strips(const T *__restrict__ data, const int64_t *__restrict__ toff,
                  const int64_t *__restrict__ voff, const int32_t *__restrict__ strip_m,
                  const int32_t *__restrict__ strip_I, const int32_t *__restrict__ cta_off,
                  const double *__restrict__ x, double *__restrict__ rowpart,
                  typename Acc<T>::type *__restrict__ colpart, int *err) {
  constexpr int R = kTile / WARPS;  // rows per warp
  static_assert(D <= NST && D * kTile <= WARPS * 32, "batch must fit the stages and the block");
  using A = typename Acc<T>::type;
  using V2 = typename Vec2<T>::type;
  extern __shared__ __align__(128) unsigned char smraw[];
  T *stage = reinterpret_cast<T *>(smraw);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smraw + (size_t)NST * kTileElems * sizeof(T));
  A *red = reinterpret_cast<A *>(bar + NST);  // [D][WARPS][64]
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const int s0 = cta_off[blockIdx.x], s1 = cta_off[blockIdx.x + 1];
  if (s0 >= s1) return;
  if (tid == 0) {
    for (int i = 0; i < NST; ++i) mbar_init(&bar[i], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // producer state (thread 0)
  int ps = s0, pJ = 0;
  long long issued = 0, consumed = 0;
  auto issue = [&]() {
    if (ps >= s1) return;
    const int m = strip_m[ps], I = strip_I[ps];
    const T *src = data + (toff[m] + (int64_t)I * (I + 1) / 2 + pJ) * kTileElems;
    const int st = (int)(issued % NST);
    fence_proxy_async();
    mbar_expect_tx(&bar[st], kTileElems * sizeof(T));
    bulk_g2s(stage + (size_t)st * kTileElems, src, kTileElems * sizeof(T), &bar[st]);
    ++issued;
    if (++pJ > I) {
      pJ = 0;
      ++ps;
    }
  };
  if (tid == 0)
    for (int q = 0; q < NST; ++q) issue();
  bool failed = false;
  for (int s = s0; s < s1 && !failed; ++s) {
    const int m = strip_m[s], I = strip_I[s];
    const int64_t vb = voff[m];
    const int64_t tb = toff[m] + (int64_t)I * (I + 1) / 2;
    A xi[R], rp[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      xi[r] = (A)x[vb + (int64_t)I * kTile + w * R + r];
      rp[r] = (A)0;
    }
    for (int J0 = 0; J0 <= I; J0 += D) {
      const int nb = min(D, I + 1 - J0);
      // x of the batch's columns, loaded before the waits
      A xj[D][2];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int64_t c = vb + (int64_t)(J0 + d) * kTile + 2 * l;
        xj[d][0] = d < nb ? (A)x[c] : (A)0;
        xj[d][1] = d < nb ? (A)x[c + 1] : (A)0;
      }
      bool ok = true;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if (d >= nb) break;
        const long long q = consumed + d;
        ok = ok && mbar_wait_bounded(&bar[(int)(q % NST)], (uint32_t)((q / NST) & 1));
      }
      // uniform decision; also orders the previous batch's red[] reads
      // before this batch's writes
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicCAS(err, kDevOk, kDevTimeout);
        failed = true;
        break;
      }
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if (d < nb) {
          const T *t = stage + (size_t)((consumed + d) % NST) * kTileElems;
          A c0 = 0, c1 = 0;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const V2 a = *reinterpret_cast<const V2 *>(t + (w * R + r) * kTile + 2 * l);
            rp[r] = fma((A)a.x, xj[d][0], fma((A)a.y, xj[d][1], rp[r]));
            c0 = fma((A)a.x, xi[r], c0);
            c1 = fma((A)a.y, xi[r], c1);
          }
          red[(d * WARPS + w) * kTile + 2 * l] = c0;
          red[(d * WARPS + w) * kTile + 2 * l + 1] = c1;
        }
      }
      __syncthreads();
      {
        const int d = tid >> 6, c = tid & 63;
        // column partials of the off-diagonal tiles (the diagonal tile is
        // stored in full and counted by the row partials)
        if (d < nb && J0 + d < I) {
          A sum = 0;
#pragma unroll
          for (int q = 0; q < WARPS; ++q) sum += red[(d * WARPS + q) * kTile + c];
          colpart[(tb + J0 + d) * kTile + c] = sum;  // in the accumulation type
        }
      }
      consumed += nb;
      if (tid == 0)
        for (int d = 0; d < nb; ++d) issue();
    }
    if (failed) break;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      A v = rp[r];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (l == 0) rowpart[vb + (int64_t)I * kTile + w * R + r] = (double)v;
    }
  }
  if (failed && tid == 0) {
    // drain copies still in flight before leaving (bounded)
    while (consumed < issued) {
      const int st = (int)(consumed % NST);
      mbar_wait_bounded(&bar[st], (uint32_t)((consumed / NST) & 1));
      ++consumed;
    }
  }
}

// The same stream for NR right-hand sides at once (float32 tiles): every
// tile is read once and applied to the NR columns x_c = x + c vlen.  For
// each column, every product and sum is formed in the order of
// k_symv_strips<float, *, *, WARPS>, so column c equals that kernel's result
// bit for bit.  Row partials go to rowpart[c][vlen], column partials to
// colpart[c][ntiles][64].
template <int NST, int D, int WARPS, int NR>
__global__ void __launch_bounds__(WARPS * 32)
    k_symv_strips_nr(const float *__restrict__ data, const int64_t *__restrict__ toff,
                     const int64_t *__restrict__ voff, const int32_t *__restrict__ strip_m,
                     const int32_t *__restrict__ strip_I, const int32_t *__restrict__ cta_off,
                     const double *__restrict__ x, int64_t vlen, int64_t ntiles,
                     double *__restrict__ rowpart, float *__restrict__ colpart, int *err) {
  constexpr int R = kTile / WARPS;  // rows per warp
  static_assert(D <= NST && D * kTile <= WARPS * 32, "batch must fit the stages and the block");
  extern __shared__ __align__(128) unsigned char smraw[];
  float *stage = reinterpret_cast<float *>(smraw);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smraw + (size_t)NST * kTileElems * sizeof(float));
  float *red = reinterpret_cast<float *>(bar + NST);  // [D][NR][WARPS][64]
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const int s0 = cta_off[blockIdx.x], s1 = cta_off[blockIdx.x + 1];
  if (s0 >= s1) return;
  if (tid == 0) {
    for (int i = 0; i < NST; ++i) mbar_init(&bar[i], 1);
    fence_mbar_init();
  }
  __syncthreads();
  int ps = s0, pJ = 0;
  long long issued = 0, consumed = 0;
  auto issue = [&]() {
    if (ps >= s1) return;
    const int m = strip_m[ps], I = strip_I[ps];
    const float *src = data + (toff[m] + (int64_t)I * (I + 1) / 2 + pJ) * kTileElems;
    const int st = (int)(issued % NST);
    fence_proxy_async();
    mbar_expect_tx(&bar[st], kTileElems * sizeof(float));
    bulk_g2s(stage + (size_t)st * kTileElems, src, kTileElems * sizeof(float), &bar[st]);
    ++issued;
    if (++pJ > I) {
      pJ = 0;
      ++ps;
    }
  };
  if (tid == 0)
    for (int q = 0; q < NST; ++q) issue();
  bool failed = false;
  for (int s = s0; s < s1 && !failed; ++s) {
    const int m = strip_m[s], I = strip_I[s];
    const int64_t vb = voff[m];
    const int64_t tb = toff[m] + (int64_t)I * (I + 1) / 2;
    float xi[R][NR], rp[R][NR];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        xi[r][c] = (float)x[c * vlen + vb + (int64_t)I * kTile + w * R + r];
        rp[r][c] = 0.0f;
      }
    for (int J0 = 0; J0 <= I; J0 += D) {
      const int nb = min(D, I + 1 - J0);
      float xj[D][2][NR];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int64_t e = vb + (int64_t)(J0 + d) * kTile + 2 * l;
#pragma unroll
        for (int c = 0; c < NR; ++c) {
          xj[d][0][c] = d < nb ? (float)x[c * vlen + e] : 0.0f;
          xj[d][1][c] = d < nb ? (float)x[c * vlen + e + 1] : 0.0f;
        }
      }
      bool ok = true;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if (d >= nb) break;
        const long long q = consumed + d;
        ok = ok && mbar_wait_bounded(&bar[(int)(q % NST)], (uint32_t)((q / NST) & 1));
      }
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicCAS(err, kDevOk, kDevTimeout);
        failed = true;
        break;
      }
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if (d < nb) {
          const float *t = stage + (size_t)((consumed + d) % NST) * kTileElems;
          float c0[NR], c1[NR];
#pragma unroll
          for (int c = 0; c < NR; ++c) c0[c] = c1[c] = 0.0f;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float2 a = *reinterpret_cast<const float2 *>(t + (w * R + r) * kTile + 2 * l);
#pragma unroll
            for (int c = 0; c < NR; ++c) {
              rp[r][c] = fmaf(a.x, xj[d][0][c], fmaf(a.y, xj[d][1][c], rp[r][c]));
              c0[c] = fmaf(a.x, xi[r][c], c0[c]);
              c1[c] = fmaf(a.y, xi[r][c], c1[c]);
            }
          }
#pragma unroll
          for (int c = 0; c < NR; ++c) {
            red[((d * NR + c) * WARPS + w) * kTile + 2 * l] = c0[c];
            red[((d * NR + c) * WARPS + w) * kTile + 2 * l + 1] = c1[c];
          }
        }
      }
      __syncthreads();
      // column partials of the off-diagonal tiles, per column
      for (int e = tid; e < D * NR * kTile; e += WARPS * 32) {
        const int d = e / (NR * kTile), c = (e / kTile) % NR, j = e % kTile;
        if (d < nb && J0 + d < I) {
          float sum = 0.0f;
#pragma unroll
          for (int q = 0; q < WARPS; ++q) sum += red[((d * NR + c) * WARPS + q) * kTile + j];
          colpart[(c * ntiles + tb + J0 + d) * kTile + j] = sum;
        }
      }
      consumed += nb;
      if (tid == 0)
        for (int d = 0; d < nb; ++d) issue();
    }
    if (failed) break;
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        float v = rp[r][c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (l == 0) rowpart[c * vlen + vb + (int64_t)I * kTile + w * R + r] = (double)v;
      }
  }
  if (failed && tid == 0) {
    while (consumed < issued) {
      const int st = (int)(consumed % NST);
      mbar_wait_bounded(&bar[st], (uint32_t)((consumed / NST) & 1));
      ++consumed;
    }
  }
}

// y[(m, I)] = rowpart[(m, I)] + sum_{K > I} colpart[(m, K, I)]; the column
// partials are stored in the accumulation type of the SYMV (float for
// float32 tiles: half the partial-sum traffic, no precision lost)
template <typename P>
__global__ void k_symv_reduce(const int32_t *__restrict__ vrow_m,
                              const int32_t *__restrict__ vrow_I, const int32_t *__restrict__ nt,
                              const int64_t *__restrict__ toff, const int64_t *__restrict__ voff,
                              const double *__restrict__ rowpart,
                              const P *__restrict__ colpart, double *__restrict__ y,
                              int64_t nblocks) {
  const int64_t blk = blockIdx.x;
  if (blk >= nblocks) return;
  const int m = vrow_m[blk], I = vrow_I[blk];
  const int r = threadIdx.x;
  const int64_t pos = voff[m] + (int64_t)I * kTile + r;
  double v = rowpart[pos];
  const int ntm = nt[m];
  for (int K = I + 1; K < ntm; ++K)
    v += (double)colpart[(toff[m] + (int64_t)K * (K + 1) / 2 + I) * kTile + r];
  y[pos] = v;
}

// Candidate launch configurations of the streaming SYMV (the autotuner's
// knob space): bulk-copy stages, tiles per barrier pair, warps per CTA and
// persistent CTAs per SM.  Entry 0 of each list is the default.
template <typename T> struct SymvCands;
template <> struct SymvCands<float> {
  static constexpr int n = 6;
  static constexpr SymvCfg c[n] = {{8, 4, 8, 1}, {8, 4, 16, 1}, {12, 4, 16, 1},
                                   {8, 8, 16, 1}, {6, 4, 8, 2}, {4, 2, 8, 2}};
};
template <> struct SymvCands<double> {
  static constexpr int n = 5;
  static constexpr SymvCfg c[n] = {{4, 2, 8, 1}, {4, 2, 16, 1}, {6, 2, 16, 1},
                                   {4, 4, 16, 1}, {3, 2, 8, 2}};
};

template <typename T, int NST, int D, int WARPS>
static void launch_symv(TileBatch &b, const TileBatch::Sched &sc, const T *data, const double *x,
                        int *d_err, cudaStream_t s) {
  const size_t smem = (size_t)NST * kTileElems * sizeof(T) + NST * sizeof(uint64_t) +
                      (size_t)D * WARPS * kTile * sizeof(typename Acc<T>::type);
  static int attr_dev = -1;
  int dev = 0;
  GENEO_CUDA(cudaGetDevice(&dev));
  if (attr_dev != dev) {
    GENEO_CUDA(cudaFuncSetAttribute(k_symv_strips<T, NST, D, WARPS>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_dev = dev;
  }
  k_symv_strips<T, NST, D, WARPS><<<sc.nctas, WARPS * 32, smem, s>>>(
      data, b.d_toff.p, b.d_voff.p, sc.strip_m.p, sc.strip_I.p, sc.cta_off.p, x, b.rowpart.p,
      reinterpret_cast<typename Acc<T>::type *>(b.colpart.p), d_err);
}

template <typename T>
static void launch_symv_cfg(TileBatch &b, int idx, const T *data, const double *x, int *d_err,
                            cudaStream_t s);
template <>
void launch_symv_cfg<float>(TileBatch &b, int idx, const float *data, const double *x,
                            int *d_err, cudaStream_t s) {
  const SymvCfg &c = SymvCands<float>::c[idx];
  const TileBatch::Sched &sc = b.sched_for(c.cps);
  switch (idx) {
    case 0: launch_symv<float, 8, 4, 8>(b, sc, data, x, d_err, s); break;
    case 1: launch_symv<float, 8, 4, 16>(b, sc, data, x, d_err, s); break;
    case 2: launch_symv<float, 12, 4, 16>(b, sc, data, x, d_err, s); break;
    case 3: launch_symv<float, 8, 8, 16>(b, sc, data, x, d_err, s); break;
    case 4: launch_symv<float, 6, 4, 8>(b, sc, data, x, d_err, s); break;
    default: launch_symv<float, 4, 2, 8>(b, sc, data, x, d_err, s); break;
  }
}
template <>
void launch_symv_cfg<double>(TileBatch &b, int idx, const double *data, const double *x,
                             int *d_err, cudaStream_t s) {
  const SymvCfg &c = SymvCands<double>::c[idx];
  const TileBatch::Sched &sc = b.sched_for(c.cps);
  switch (idx) {
    case 0: launch_symv<double, 4, 2, 8>(b, sc, data, x, d_err, s); break;
    case 1: launch_symv<double, 4, 2, 16>(b, sc, data, x, d_err, s); break;
    case 2: launch_symv<double, 6, 2, 16>(b, sc, data, x, d_err, s); break;
    case 3: launch_symv<double, 4, 4, 16>(b, sc, data, x, d_err, s); break;
    default: launch_symv<double, 3, 2, 8>(b, sc, data, x, d_err, s); break;
  }
}

template <typename T> int symv_candidates() { return SymvCands<T>::n; }
template <typename T> SymvCfg symv_candidate(int idx) { return SymvCands<T>::c[idx]; }
template int symv_candidates<float>();
template int symv_candidates<double>();
template SymvCfg symv_candidate<float>(int);
template SymvCfg symv_candidate<double>(int);

template <typename T>
void symv_batch(TileBatch &b, const T *data, const double *x, double *y, int *d_err,
                cudaStream_t s, cudaEvent_t ev_before, cudaEvent_t ev_after) {
  const int idx = b.symv_cfg[sizeof(T) == 8 ? 1 : 0];
  if (ev_before) record_event(ev_before, s);
  launch_symv_cfg<T>(b, idx, data, x, d_err, s);
  if (ev_after) record_event(ev_after, s);
  const int64_t nblocks = b.vlen / kTile;
  k_symv_reduce<<<(unsigned)nblocks, kTile, 0, s>>>(b.d_vrow_m.p, b.d_vrow_I.p, b.d_nt.p,
                                                    b.d_toff.p, b.d_voff.p, b.rowpart.p,
                                                    reinterpret_cast<const typename Acc<T>::type *>(b.colpart.p),
                                                    y, nblocks);
  GENEO_CHECK_LAUNCH();
}

template <int NST, int D, int WARPS>
static void launch_symv_nr4(TileBatch &b, const TileBatch::Sched &sc, const float *data,
                            const double *x, int *d_err, cudaStream_t s) {
  constexpr int NR = 4;
  const size_t smem = (size_t)NST * kTileElems * sizeof(float) + NST * sizeof(uint64_t) +
                      (size_t)D * NR * WARPS * kTile * sizeof(float);
  static int attr_dev = -1;
  int dev = 0;
  GENEO_CUDA(cudaGetDevice(&dev));
  if (attr_dev != dev) {
    GENEO_CUDA(cudaFuncSetAttribute(k_symv_strips_nr<NST, D, WARPS, NR>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_dev = dev;
  }
  k_symv_strips_nr<NST, D, WARPS, NR><<<sc.nctas, WARPS * 32, smem, s>>>(
      data, b.d_toff.p, b.d_voff.p, sc.strip_m.p, sc.strip_I.p, sc.cta_off.p, x, b.vlen,
      b.ntiles, b.rowpart_nr.p, b.colpart_nr.p, d_err);
}

void symv_batch_f32_cols(TileBatch &b, const float *data, const double *x, double *y, int nr,
                         int *d_err, cudaStream_t s, cudaEvent_t ev_before,
                         cudaEvent_t ev_after) {
  constexpr int NR = 4;
  // the warps per tile of the batch's float configuration fix the order of
  // every sum, so the 4-column kernel takes the same
  const int warps = SymvCands<float>::c[b.symv_cfg[0]].warps;
  int c = 0;
  if (nr >= NR) {
    if (b.rowpart_nr.n < b.vlen * NR) b.rowpart_nr.alloc(b.vlen * NR);
    if (b.colpart_nr.n < b.ntiles * (int64_t)kTile * NR) b.colpart_nr.alloc(b.ntiles * kTile * NR);
  }
  const int64_t nblocks = b.vlen / kTile;
  for (; c + NR <= nr; c += NR) {
    const double *xc = x + (int64_t)c * b.vlen;
    if (c == 0 && ev_before) record_event(ev_before, s);
    if (warps == 8) launch_symv_nr4<4, 2, 8>(b, b.sched_for(2), data, xc, d_err, s);
    else launch_symv_nr4<4, 2, 16>(b, b.sched_for(1), data, xc, d_err, s);
    if (c == 0 && ev_after) record_event(ev_after, s);
    for (int q = 0; q < NR; ++q)
      k_symv_reduce<<<(unsigned)nblocks, kTile, 0, s>>>(
          b.d_vrow_m.p, b.d_vrow_I.p, b.d_nt.p, b.d_toff.p, b.d_voff.p,
          b.rowpart_nr.p + (int64_t)q * b.vlen, b.colpart_nr.p + (int64_t)q * b.ntiles * kTile,
          y + (int64_t)(c + q) * b.vlen, nblocks);
    GENEO_CHECK_LAUNCH();
  }
  for (; c < nr; ++c)
    symv_batch<float>(b, data, x + (int64_t)c * b.vlen, y + (int64_t)c * b.vlen, d_err, s);
}

template void symv_batch<double>(TileBatch &, const double *, const double *, double *, int *,
                                 cudaStream_t, cudaEvent_t, cudaEvent_t);
template void symv_batch<float>(TileBatch &, const float *, const double *, double *, int *,
                                cudaStream_t, cudaEvent_t, cudaEvent_t);

}  // namespace geneo
