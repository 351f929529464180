// Solve path: CSR SpMV, restriction, batched local solves, prolongation,
// coarse correction and preconditioned CG, all on one stream.
//
// Preconditioner (Sec. 2, eq. "AS2"; closed form at the end of Sec. 3.2):
//   y0 = Z E^-1 Z^T r ;  s = r - A y0 ;  w = sum_i R_i^T A_i^-1 R_i s ;
//   z  = y0 + w - Z E^-1 Z^T (A w).
// PCG: A is SPD (Sec. 2) and M^-1_AS,2 symmetric (eq. "AS2").
//
// Balanced form (optional): PCG starts from x0 = Z E^-1 Z^T b, so that
// Z^T r_k = 0 in exact arithmetic, and applies
//   w = sum_i R_i^T A_i^-1 R_i r ;  z = w + Z E^-1 Z^T (r - A w),
// the same operator on such residuals with one coarse solve per apply
// instead of two (the Z E^-1 Z^T r part of the added term corrects the
// rounding drift of Z^T r_k).
#include <algorithm>
#include <chrono>

#include "setup.hpp"

namespace geneo {

// Sliced ELLPACK SpMV (SELL-32-256): rows sorted by decreasing length
// within windows of 256, slices of 32 sorted rows stored column-major
// (entry j of the slice's row t at slice_off + 32 j + t), each slice padded
// to its longest row with zero values; one thread per sorted row, so every
// load of values and column indices is one coalesced 256 / 128-byte access
// per warp.  perm maps sorted positions to rows.  y = A x, or y = b - A x
// when b is given.
__global__ void __launch_bounds__(256)
    k_spmv_sell(const int64_t *__restrict__ slice_off, const int32_t *__restrict__ slice_w,
                const int32_t *__restrict__ col, const double *__restrict__ val,
                const int32_t *__restrict__ perm, const double *__restrict__ x,
                const double *__restrict__ b, double *__restrict__ y, int64_t n,
                int64_t nslices) {
  x += blockIdx.y * n;
  y += blockIdx.y * n;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t sl = t >> 5;
  if (sl >= nslices) return;
  const int lane = threadIdx.x & 31;
  const int64_t base = slice_off[sl] + lane;
  const int w = slice_w[sl];
  double acc = 0;
  // chunks of 8 entries: the values and indices (streamed, not kept in L1)
  // are loaded first, then the 8 gathers of x, so that each thread has 8
  // independent loads in flight at every stage; the sum keeps the entry order
  for (int j0 = 0; j0 < w; j0 += 8) {
    double v[8], xv[8];
    int32_t ci[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (j0 + q < w) {
        const int64_t e = base + (int64_t)(j0 + q) * 32;
        v[q] = __ldcs(val + e);
        ci[q] = __ldcs(col + e);
      }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (j0 + q < w) xv[q] = __ldg(x + ci[q]);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (j0 + q < w) acc = fma(v[q], xv[q], acc);
  }
  const int64_t i = sl * 32 + lane;
  if (i < n) {
    const int32_t r = perm[i];
    y[r] = b ? b[blockIdx.y * n + r] - acc : acc;
  }
}

// SELL value gather from the CSR values (padding slots keep 0)
__global__ void k_sell_fill(const int64_t *__restrict__ pos, const double *__restrict__ csr,
                            double *__restrict__ sell, int64_t nnz) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < nnz) sell[pos[k]] = csr[k];
}

// padded local vector x_loc[p] = s[l2g[p]] (0 on padding)
__global__ void k_restrict(const int32_t *__restrict__ l2g, const double *__restrict__ s,
                           double *__restrict__ xl, int64_t len, int64_t n) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= len) return;
  s += blockIdx.y * n;
  xl += blockIdx.y * len;
  const int32_t g = l2g[p];
  xl[p] = g >= 0 ? s[g] : 0.0;
}

// w[e] = sum over the local slots holding e (deterministic gather-sum)
__global__ void k_prolong(const int64_t *__restrict__ ptr, const int64_t *__restrict__ slot,
                          const double *__restrict__ yl, double *__restrict__ w, int64_t n,
                          int64_t len) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  yl += blockIdx.y * len;
  w += blockIdx.y * n;
  double s = 0;
  for (int64_t k = ptr[e]; k < ptr[e + 1]; ++k) s += yl[slot[k]];
  w[e] = s;
}

// t[a] = (Z^T r)_a, one column per warp (CSC): split near-kernel columns
// have a few entries, GenEO columns one per dof of their subdomain
__global__ void k_zt(const int64_t *__restrict__ zptr, const int32_t *__restrict__ zrow,
                     const double *__restrict__ zval, const double *__restrict__ r,
                     double *__restrict__ t, int64_t ncols, int64_t n0, int64_t n) {
  const int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int l = threadIdx.x & 31;
  if (a >= ncols) return;
  r += blockIdx.y * n;
  t += blockIdx.y * n0;
  double s = 0;
  for (int64_t k = zptr[a] + l; k < zptr[a + 1]; k += 32) s = fma(zval[k], r[zrow[k]], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (l == 0) t[a] = s;
}

// t[a] = (Z^T r)_a for the long columns a >= a0 (the GenEO columns, one
// entry per dof of their subdomain): one CTA per column
__global__ void k_zt_long(const int64_t *__restrict__ zptr, const int32_t *__restrict__ zrow,
                          const double *__restrict__ zval, const double *__restrict__ r,
                          double *__restrict__ t, int64_t a0, int64_t n0, int64_t n) {
  const int64_t a = a0 + blockIdx.x;
  r += blockIdx.y * n;
  t += blockIdx.y * n0;
  double s = 0;
  for (int64_t k = zptr[a] + threadIdx.x; k < zptr[a + 1]; k += blockDim.x)
    s = fma(zval[k], r[zrow[k]], s);
  __shared__ double sh[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[w];
    t[a] = v;
  }
}

// y[e] = (Z u)_e (+ add[e] when add is given), one row per thread (CSR)
__global__ void k_z(const int64_t *__restrict__ zptr, const int32_t *__restrict__ zcol,
                    const double *__restrict__ zval, const double *__restrict__ u,
                    double *__restrict__ y, int64_t n, int64_t n0,
                    const double *__restrict__ add) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  u += blockIdx.y * n0;
  y += blockIdx.y * n;
  double s = 0;
  for (int64_t k = zptr[e]; k < zptr[e + 1]; ++k) s = fma(zval[k], u[zcol[k]], s);
  y[e] = add ? add[blockIdx.y * n + e] + s : s;
}

// Error-free transformations for the accurate residual (Dot2 of Ogita, Rump
// and Oishi, SIAM J. Sci. Comput. 26, 2005): a*b = p + e exactly with
// p = fl(a*b), e = fma(a, b, -p); a + b = s + t exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &t) {
  s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  t = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

// y = b - A x as accurately as if computed in twice the working precision,
// then rounded to float64; 8 lanes per row
__global__ void k_residual_dd(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                              const double *__restrict__ val, const double *__restrict__ x,
                              const double *__restrict__ b, double *__restrict__ y, int64_t n) {
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gt >> 3;
  const int lane = threadIdx.x & 7;
  double hi = 0, lo = 0;
  if (row < n)
    for (int32_t k = rowptr[row] + lane; k < rowptr[row + 1]; k += 8) {
      const double a = val[k], v = x[col[k]];
      const double p = __dmul_rn(a, v);
      const double pe = fma(a, v, -p);
      double t;
      two_sum(hi, p, hi, t);
      lo = __dadd_rn(lo, __dadd_rn(t, pe));
    }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    const double ohi = __shfl_xor_sync(0xffffffffu, hi, o);
    const double olo = __shfl_xor_sync(0xffffffffu, lo, o);
    double t;
    two_sum(hi, ohi, hi, t);
    lo = __dadd_rn(lo, __dadd_rn(olo, t));
  }
  if (row < n && lane == 0) {
    double sres, t;
    two_sum(b[row], -hi, sres, t);
    y[row] = __dadd_rn(sres, __dsub_rn(t, lo));
  }
}

// x += d
__global__ void k_axpy1(const double *__restrict__ d, double *__restrict__ x, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] += d[i];
}

// z = y0 + w - c
__global__ void k_combine(const double *__restrict__ y0, const double *__restrict__ w,
                          const double *__restrict__ c, double *__restrict__ z, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t o = blockIdx.y * n;
  if (i < n) z[o + i] = (y0[o + i] + w[o + i]) - c[o + i];
}

// ---------------------------------------------------------------------------
// deterministic dot products: fixed grid, block partials, one final block

constexpr int kDotBlocks = 512;
constexpr int kScal = 8;  // PCG scalars per right-hand side

__global__ void k_dot_partial(const double *__restrict__ a, const double *__restrict__ b, int64_t n,
                              double *__restrict__ part) {
  __shared__ double sh[256];
  a += blockIdx.y * n;
  b += blockIdx.y * n;
  part += blockIdx.y * gridDim.x;
  double s = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

// one block per column; out[column * kScal]
__global__ void k_dot_final(const double *__restrict__ part, int np, double *__restrict__ out) {
  __shared__ double sh[32];
  part += blockIdx.x * np;
  out += blockIdx.x * kScal;
  double s = 0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = s;
  }
}

static void dot(geneo_ctx *c, const double *a, const double *b, int64_t n, double *out,
                cudaStream_t s, int k = 1) {
  c->launches += 2;
  k_dot_partial<<<dim3(kDotBlocks, k), 256, 0, s>>>(a, b, n, c->partials.p);
  k_dot_final<<<k, 256, 0, s>>>(c->partials.p, kDotBlocks, out);
}
// scalars per column c at sc[c * kScal]: 0 rz, 1 pq, 2 rr, 3 rz_new, 4 bb;
// act[c] = 0 freezes a converged column
// x += alpha p ; r -= alpha q  with alpha = rz / pq
__global__ void k_update_xr(const double *__restrict__ sc, const int *__restrict__ act,
                            const double *__restrict__ p, const double *__restrict__ q,
                            double *__restrict__ x, double *__restrict__ r, int64_t n) {
  if (!act[blockIdx.y]) return;
  sc += blockIdx.y * kScal;
  const int64_t o = blockIdx.y * n;
  const double alpha = sc[0] / sc[1];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    x[o + i] = fma(alpha, p[o + i], x[o + i]);
    r[o + i] = fma(-alpha, q[o + i], r[o + i]);
  }
}

// p = z + beta p with beta = rz_new / rz
__global__ void k_update_p(const double *__restrict__ sc, const int *__restrict__ act,
                           const double *__restrict__ z, double *__restrict__ p, int64_t n) {
  if (!act[blockIdx.y]) return;
  sc += blockIdx.y * kScal;
  const int64_t o = blockIdx.y * n;
  const double beta = sc[3] / sc[0];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[o + i] = fma(beta, p[o + i], z[o + i]);
}

// rz = rz_new, one thread per column
__global__ void k_shift_rz(double *sc, int k) {
  const int c = threadIdx.x;
  if (c < k) sc[c * kScal] = sc[c * kScal + 3];
}

__global__ void k_copy(const double *__restrict__ a, double *__restrict__ b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t o = blockIdx.y * n;
  if (i < n) b[o + i] = a[o + i];
}

// ---------------------------------------------------------------------------
// Work buffers for k right-hand-side columns (column c of a vector of length
// len at offset c * len).  Growing them invalidates the captured graph.

void reserve_rhs(geneo_ctx *c, int k) {
  if (k <= c->kcap) return;
  c->drop_graph();
  cudaStream_t s = c->stream;
  const int64_t n = c->topo.ndofs();
  for (auto *v : {&c->v_y0, &c->v_s, &c->v_w, &c->v_t, &c->v_c, &c->p_r, &c->p_z, &c->p_p,
                  &c->p_q, &c->p_x})
    v->alloc(n * k);
  c->loc_x.alloc(c->loc.vlen * k);
  c->loc_y.alloc(c->loc.vlen * k);
  if (c->tc) {
    c->loc_xp.alloc(c->loc.vlen * k);
    c->loc_xp.zero(s);  // padding rows stay zero
  }
  if (c->n0 > 0) {
    const int64_t len = c->mf ? c->n0 : c->crs.vlen;
    c->crs_x.alloc(len * k);
    c->crs_y.alloc(len * k);
    c->crs_x.zero(s);
    if (c->mf) mf_reserve(c, k);
  }
  if (c->xi) {
    for (auto *u : {&c->xi->u1, &c->xi->u2, &c->xi->u3}) {
      u->alloc(c->xi->vlenS * k);
      u->zero(s);
    }
  }
  c->scal.alloc((int64_t)kScal * k);
  c->scal.zero(s);
  c->partials.alloc((int64_t)kDotBlocks * k);
  c->d_act.alloc(k);
  if (c->h_scal) GENEO_CUDA(cudaFreeHost(c->h_scal));
  c->h_scal = nullptr;
  GENEO_CUDA(cudaMallocHost((void **)&c->h_scal, sizeof(double) * kScal * k));
  if (c->h_act) GENEO_CUDA(cudaFreeHost(c->h_act));
  c->h_act = nullptr;
  GENEO_CUDA(cudaMallocHost((void **)&c->h_act, sizeof(int) * k));
  GENEO_CUDA(cudaStreamSynchronize(s));
  c->kcap = k;
}

// Builds the SELL-32-256 copy of A from the CSR pattern (host) and values
// (device gather).
void build_sell(geneo_ctx *c, cudaStream_t s) {
  const Topology &t = c->topo;
  const int64_t n = t.ndofs(), nnz = t.nnz();
  constexpr int C = 32, SIGMA = 256;
  std::vector<int32_t> perm(n);
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  auto len = [&](int32_t r) { return t.rowptr[r + 1] - t.rowptr[r]; };
  for (int64_t w0 = 0; w0 < n; w0 += SIGMA) {
    const int64_t w1 = std::min<int64_t>(n, w0 + SIGMA);
    std::stable_sort(perm.begin() + w0, perm.begin() + w1,
                     [&](int32_t a, int32_t b) { return len(a) > len(b); });
  }
  const int64_t nsl = (n + C - 1) / C;
  std::vector<int64_t> off(nsl + 1, 0);
  std::vector<int32_t> wid(nsl, 0);
  for (int64_t sl = 0; sl < nsl; ++sl) {
    int w = 0;
    for (int64_t i = sl * C; i < std::min<int64_t>(n, (sl + 1) * C); ++i) w = std::max(w, (int)len(perm[i]));
    wid[sl] = w;
    off[sl + 1] = off[sl] + (int64_t)w * C;
  }
  std::vector<int32_t> col(off[nsl]);
  std::vector<int64_t> pos(nnz);
  for (int64_t sl = 0; sl < nsl; ++sl)
    for (int lane = 0; lane < C; ++lane) {
      const int64_t i = sl * C + lane;
      const int32_t r = i < n ? perm[i] : -1;
      for (int j = 0; j < wid[sl]; ++j) {
        const int64_t q = off[sl] + (int64_t)j * C + lane;
        if (r >= 0 && j < len(r)) {
          col[q] = t.col[t.rowptr[r] + j];
          pos[t.rowptr[r] + j] = q;
        } else {
          col[q] = r >= 0 ? r : 0;  // padding: a valid column, value 0
        }
      }
    }
  c->sell_nslices = nsl;
  c->sell_stored = off[nsl];
  c->d_sell_off.upload(off, s);
  c->d_sell_w.upload(wid, s);
  c->d_sell_col.upload(col, s);
  c->d_sell_perm.upload(perm, s);
  c->d_sell_val.alloc(off[nsl]);
  c->d_sell_val.zero(s);
  DevBuf<int64_t> dpos;
  dpos.upload(pos, s);
  k_sell_fill<<<grid_for(nnz, 256), 256, 0, s>>>(dpos.p, c->d_val.p, c->d_sell_val.p, nnz);
  GENEO_CHECK_LAUNCH();
  GENEO_CUDA(cudaStreamSynchronize(s));
}

static void sell_apply(geneo_ctx *c, const double *x, const double *b, double *y, cudaStream_t s,
                       int k) {
  const int64_t n = c->topo.ndofs();
  c->launches += 1;
  k_spmv_sell<<<dim3(grid_for(c->sell_nslices * 32, 256), k), 256, 0, s>>>(
      c->d_sell_off.p, c->d_sell_w.p, c->d_sell_col.p, c->d_sell_val.p, c->d_sell_perm.p, x, b,
      y, n, c->sell_nslices);
  GENEO_CHECK_LAUNCH();
}

void spmv(geneo_ctx *c, const double *x, double *y, cudaStream_t s, int k) {
  sell_apply(c, x, nullptr, y, s, k);
}

// y = b - A x (k columns)
void residual(geneo_ctx *c, const double *x, const double *b, double *y, cudaStream_t s,
                     int k) {
  sell_apply(c, x, b, y, s, k);
}

void local_solve(geneo_ctx *c, const double *r, double *w, cudaStream_t s, int k) {
  const int64_t n = c->topo.ndofs(), vlen = c->loc.vlen;
  c->launches += 2;
  k_restrict<<<dim3(grid_for(vlen, 256), k), 256, 0, s>>>(c->d_l2g.p, r, c->loc_x.p, vlen, n);
  if (c->local_prec == GENEO_PREC_BF16) {
    // tensor cores: every column in one pass over the bfloat16 factors
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->prof) {
      e0 = c->ev_take();
      e1 = c->ev_take();
      c->ev_local.push_back({e0, e1});
    }
    c->launches += 6 + 4 * k;
    split_tc_apply(c, c->loc_x.p, c->loc_y.p, c->loc_xp.p, s, k, e0, e1);
    k_prolong<<<dim3(grid_for(n, 256), k), 256, 0, s>>>(c->d_g2l_ptr.p, c->d_g2l.p, c->loc_y.p, w,
                                                        n, vlen);
    GENEO_CHECK_LAUNCH();
    return;
  }
  for (int j = 0; j < k;) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->prof) {
      e0 = c->ev_take();
      e1 = c->ev_take();
      c->ev_local.push_back({e0, e1});
    }
    const double *xj = c->loc_x.p + j * vlen;
    double *yj = c->loc_y.p + j * vlen;
    if (c->local_prec == GENEO_PREC_FP32 && k - j >= 4) {
      // four columns per pass over the float32 factors (same bits per column)
      c->launches += 5;
      symv_batch_f32_cols(c->loc, c->loc_f32.p, xj, yj, 4, c->d_err.p, s, e0, e1);
      j += 4;
      continue;
    }
    c->launches += 2;
    if (c->local_prec == GENEO_PREC_FP32)
      symv_batch<float>(c->loc, c->loc_f32.p, xj, yj, c->d_err.p, s, e0, e1);
    else
      symv_batch<double>(c->loc, c->loc_f64.p, xj, yj, c->d_err.p, s, e0, e1);
    ++j;
  }
  if (c->local_prec == GENEO_PREC_FP32) {
    // split inverse: float32 C_j r_j plus the float64 gradient part
    split_gradient_apply(c, c->loc_x.p, c->loc_y.p, s, k);
    c->launches += 2 + 2 * k;
  } else if (c->xi && c->xi->shifted) {
    // shifted float64 inverse: A_j^-1 = A~_j^-1 + rho/(1+rho) G S^-1 G^T
    split_gradient_apply(c, c->loc_x.p, c->loc_y.p, s, k, c->xi->gsc64.p);
    c->launches += 2 + 2 * k;
  }
  k_prolong<<<dim3(grid_for(n, 256), k), 256, 0, s>>>(c->d_g2l_ptr.p, c->d_g2l.p, c->loc_y.p, w,
                                                      n, vlen);
  GENEO_CHECK_LAUNCH();
}

void coarse_solve(geneo_ctx *c, const double *r, double *y, cudaStream_t s, int k,
                  const double *add) {
  const int64_t n = c->topo.ndofs(), n0 = c->n0;
  if (n0 == 0) {
    if (add) GENEO_CUDA(cudaMemcpyAsync(y, add, sizeof(double) * n * k, cudaMemcpyDeviceToDevice, s));
    else GENEO_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * n * k, s));
    return;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->prof) {
    e0 = c->ev_take();
    e1 = c->ev_take();
    c->ev_coarse.push_back({e0, e1});
  }
  // short columns (split near-kernel) a warp each, long ones (GenEO) a CTA each
  const int64_t nshort = c->n0_snk, nlong = n0 - c->n0_snk;
  c->launches += 1;
  if (nshort > 0) {
    c->launches += 1;
    k_zt<<<dim3(grid_for(nshort * 32, 256), k), 256, 0, s>>>(c->d_zc_ptr.p, c->d_zc_row.p,
                                                             c->d_zc_val.p, r, c->crs_x.p, nshort,
                                                             n0, n);
  }
  if (nlong > 0) {
    c->launches += 1;
    k_zt_long<<<dim3((unsigned)nlong, k), 256, 0, s>>>(c->d_zc_ptr.p, c->d_zc_row.p,
                                                       c->d_zc_val.p, r, c->crs_x.p, nshort, n0, n);
  }
  if (c->mf) {
    c->launches += mf_launches_per_solve(c);
    if (e0) record_event(e0, s);
    mf_solve(c, c->crs_x.p, c->crs_y.p, s, k);
    if (e1) record_event(e1, s);
  } else {
    // explicit dense E^-1, one SYMV per column
    if (k != 1) throw Error(GENEO_ERR_STATE, "the dense coarse inverse solves one column at a time");
    c->launches += 2;
    symv_batch<double>(c->crs, c->crs_f64.p, c->crs_x.p, c->crs_y.p, c->d_err.p, s, e0, e1);
  }
  k_z<<<dim3(grid_for(n, 256), k), 256, 0, s>>>(c->d_zr_ptr.p, c->d_zr_col.p, c->d_zr_val.p,
                                                c->crs_y.p, y, n, n0, add);
  GENEO_CHECK_LAUNCH();
}

void apply_preconditioner(geneo_ctx *c, const double *r, double *z, cudaStream_t s, int k) {
  const int64_t n = c->topo.ndofs();
  if (c->n0 == 0) {
    local_solve(c, r, z, s, k);
    return;
  }
  c->launches += 1;
  coarse_solve(c, r, c->v_y0.p, s, k);
  residual(c, c->v_y0.p, r, c->v_s.p, s, k);
  local_solve(c, c->v_s.p, c->v_w.p, s, k);
  spmv(c, c->v_w.p, c->v_t.p, s, k);
  coarse_solve(c, c->v_t.p, c->v_c.p, s, k);
  k_combine<<<dim3(grid_for(n, 256), k), 256, 0, s>>>(c->v_y0.p, c->v_w.p, c->v_c.p, z, n);
  GENEO_CHECK_LAUNCH();
}

void apply_balanced(geneo_ctx *c, const double *r, double *z, cudaStream_t s, int k) {
  const int64_t n = c->topo.ndofs();
  if (c->n0 == 0) {
    local_solve(c, r, z, s, k);
    return;
  }
  local_solve(c, r, c->v_w.p, s, k);
  residual(c, c->v_w.p, r, c->v_t.p, s, k);
  coarse_solve(c, c->v_t.p, z, s, k, c->v_w.p);
}

// the preconditioner of the PCG iteration: literal or balanced form
static void precondition(geneo_ctx *c, const double *r, double *z, cudaStream_t s, int k) {
  if (c->balanced) apply_balanced(c, r, z, s, k);
  else apply_preconditioner(c, r, z, s, k);
}

// x0 and r0 = b - A x0: zero and b, or Z E^-1 Z^T b and its residual
static void pcg_start(geneo_ctx *c, const double *b, double *x, cudaStream_t s, int k) {
  const int64_t n = c->topo.ndofs();
  if (c->balanced && c->n0 > 0) {
    coarse_solve(c, b, x, s, k);
    residual(c, x, b, c->p_r.p, s, k);
  } else {
    GENEO_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n * k, s));
    c->launches += 1;
    k_copy<<<dim3(grid_for(n, 256), k), 256, 0, s>>>(b, c->p_r.p, n);
  }
  GENEO_CHECK_LAUNCH();
}

// second half of a PCG iteration: z = M^-1 r, rz_new = (r, z), p = z + beta p
static void pcg_precond_half(geneo_ctx *c, cudaStream_t s, int k) {
  const int64_t n = c->topo.ndofs();
  double *sc = c->scal.p;
  precondition(c, c->p_r.p, c->p_z.p, s, k);
  dot(c, c->p_r.p, c->p_z.p, n, sc + 3, s, k);
  c->launches += 2;
  k_update_p<<<dim3(grid_for(n, 256), k), 256, 0, s>>>(sc, c->d_act.p, c->p_z.p, c->p_p.p, n);
  k_shift_rz<<<1, 32, 0, s>>>(sc, k);
  GENEO_CHECK_LAUNCH();
}

// first half: q = A p, alpha = rz / (p, q), x += alpha p, r -= alpha q,
// rr = (r, r), scalars copied to the pinned host mirror
static void pcg_step_half(geneo_ctx *c, double *x, cudaStream_t s, int k) {
  const int64_t n = c->topo.ndofs();
  double *sc = c->scal.p;
  spmv(c, c->p_p.p, c->p_q.p, s, k);
  dot(c, c->p_p.p, c->p_q.p, n, sc + 1, s, k);
  c->launches += 1;
  k_update_xr<<<dim3(grid_for(n, 256), k), 256, 0, s>>>(sc, c->d_act.p, c->p_p.p, c->p_q.p, x,
                                                         c->p_r.p, n);
  dot(c, c->p_r.p, c->p_r.p, n, sc + 2, s, k);
  GENEO_CUDA(cudaMemcpyAsync(c->h_scal, sc, sizeof(double) * kScal * k, cudaMemcpyDeviceToHost, s));
  GENEO_CHECK_LAUNCH();
}

// Captures [second half ; first half] of an iteration for k columns on the
// context's capture stream, with x = p_x; replayed on the caller's stream for
// every iteration after the first.
static void ensure_pcg_graph(geneo_ctx *c, int k) {
  const int cfg = ((c->loc.symv_cfg[0] * 8 + c->loc.symv_cfg[1]) * 2 + (c->grad32 ? 1 : 0)) * 2 +
                  (c->mf_persist ? 1 : 0);
  const int key =
      (((((c->local_prec * 2 + (c->prof ? 1 : 0)) * 2 + (c->balanced ? 1 : 0)) * 256 + cfg)) << 8) + k;
  if (c->pcg_exec && c->pcg_key == key) return;
  c->drop_graph();
  const int64_t l0 = c->launches;
  const size_t nl = c->ev_local.size(), nc = c->ev_coarse.size();
  cudaStream_t cs = c->cap_stream;
  GENEO_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaGraph_t graph = nullptr;
  try {
    pcg_precond_half(c, cs, k);
    pcg_step_half(c, c->p_x.p, cs, k);
  } catch (...) {
    cudaStreamEndCapture(cs, &graph);
    if (graph) cudaGraphDestroy(graph);
    c->launches = l0;
    throw;
  }
  GENEO_CUDA(cudaStreamEndCapture(cs, &graph));
  cudaGraphExec_t exec = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  GENEO_CUDA(e);
  c->pcg_exec = exec;
  c->pcg_key = key;
  c->pcg_graph_launches = c->launches - l0;
  c->launches = l0;
  // event pairs recorded by the graph's nodes belong to the graph
  c->g_ev_local.assign(c->ev_local.begin() + nl, c->ev_local.end());
  c->ev_local.resize(nl);
  c->g_ev_coarse.assign(c->ev_coarse.begin() + nc, c->ev_coarse.end());
  c->ev_coarse.resize(nc);
}

static void harvest_graph_events(geneo_ctx *c) {
  auto add = [](std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &v, double &ms, int64_t &k) {
    for (auto &p : v) {
      float t = 0;
      GENEO_CUDA(cudaEventElapsedTime(&t, p.first, p.second));
      ms += t;
      ++k;
    }
  };
  add(c->g_ev_local, c->acc_local_ms, c->acc_local_n);
  add(c->g_ev_coarse, c->acc_coarse_ms, c->acc_coarse_n);
}

// k independent preconditioned CG iterations sharing the operator; a column
// stops (is frozen) at its own convergence.  info[c] per column.
int pcg(geneo_ctx *c, const double *b, double *x, double tol, int maxit, geneo_solve_info *info,
        cudaStream_t s, int k) {
  const auto t0 = std::chrono::steady_clock::now();
  reserve_rhs(c, k);
  const int64_t n = c->topo.ndofs();
  double *sc = c->scal.p;
  double *hs = c->h_scal;
  int *ha = c->h_act;
  const dim3 g(grid_for(n, 256), k);
  const bool graph = c->opt.use_graph != 0;
  double *xw = graph ? c->p_x.p : x;  // the graph is built on the context's own x
  pcg_start(c, b, xw, s, k);
  c->launches += 1;
  dot(c, b, b, n, sc + 4, s, k);
  precondition(c, c->p_r.p, c->p_z.p, s, k);
  k_copy<<<g, 256, 0, s>>>(c->p_z.p, c->p_p.p, n);
  dot(c, c->p_r.p, c->p_z.p, n, sc + 0, s, k);
  GENEO_CUDA(cudaMemcpyAsync(hs, sc, sizeof(double) * kScal * k, cudaMemcpyDeviceToHost, s));
  GENEO_CUDA(cudaStreamSynchronize(s));
  std::vector<double> bnorm(k), rel(k, 1.0);
  std::vector<int> st(k, GENEO_NOT_CONVERGED), its(k, 0);
  int nact = 0;
  for (int j = 0; j < k; ++j) {
    bnorm[j] = std::sqrt(hs[j * kScal + 4]);
    ha[j] = bnorm[j] > 0.0;
    if (!ha[j]) {
      st[j] = GENEO_OK;
      rel[j] = 0.0;
    }
    nact += ha[j];
  }
  GENEO_CUDA(cudaMemcpyAsync(c->d_act.p, ha, sizeof(int) * k, cudaMemcpyHostToDevice, s));
  for (int it = 1; it <= maxit && nact > 0; ++it) {
    const bool replay = graph && it > 1;
    if (it == 1) {
      pcg_step_half(c, xw, s, k);
    } else if (replay) {
      ensure_pcg_graph(c, k);
      GENEO_CUDA(cudaGraphLaunch(c->pcg_exec, s));
      c->launches += c->pcg_graph_launches;
    } else {
      pcg_precond_half(c, s, k);
      pcg_step_half(c, xw, s, k);
    }
    GENEO_CUDA(cudaStreamSynchronize(s));
    if (replay && c->prof) harvest_graph_events(c);
    bool changed = false;
    for (int j = 0; j < k; ++j) {
      if (!ha[j]) continue;
      its[j] = it;
      const double *h = hs + j * kScal;
      if (!(h[1] > 0.0) || !std::isfinite(h[1]) || !std::isfinite(h[2])) {
        st[j] = GENEO_ERR_BREAKDOWN;
      } else {
        rel[j] = std::sqrt(h[2]) / bnorm[j];
        if (rel[j] <= tol) st[j] = GENEO_OK;
      }
      if (st[j] != GENEO_NOT_CONVERGED) {
        ha[j] = 0;
        --nact;
        changed = true;
      }
    }
    if (changed && nact > 0)
      GENEO_CUDA(cudaMemcpyAsync(c->d_act.p, ha, sizeof(int) * k, cudaMemcpyHostToDevice, s));
  }
  if (xw != x) {
    c->launches += 1;
    k_copy<<<g, 256, 0, s>>>(xw, x, n);
    GENEO_CHECK_LAUNCH();
  }
  GENEO_CUDA(cudaStreamSynchronize(s));
  check_device_error(c, s);
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int status = GENEO_OK;
  for (int j = 0; j < k; ++j) {
    if (info) {
      info[j].iters = its[j];
      info[j].relres = rel[j];
      info[j].seconds = secs;
    }
    if (st[j] == GENEO_ERR_BREAKDOWN) status = GENEO_ERR_BREAKDOWN;
    else if (st[j] == GENEO_NOT_CONVERGED && status == GENEO_OK) status = GENEO_NOT_CONVERGED;
  }
  return status;
}

// ---------------------------------------------------------------------------
// Independent components (block-diagonal A, Z and M^-1): one PCG per
// component in the same launches, scalars per component.

namespace {

// out[s * kScal] = (a, b) over component s's unknowns (one CTA per component)
__global__ void k_seg_dot(const double *__restrict__ a, const double *__restrict__ b,
                          const int64_t *__restrict__ off, double *__restrict__ out) {
  __shared__ double sh[256];
  const int sg = blockIdx.x;
  double v = 0;
  for (int64_t i = off[sg] + threadIdx.x; i < off[sg + 1]; i += blockDim.x) v = fma(a[i], b[i], v);
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(int64_t)sg * kScal] = sh[0];
}

__global__ void k_seg_update_xr(const double *__restrict__ sc, const int *__restrict__ act,
                                const int32_t *__restrict__ seg, const double *__restrict__ p,
                                const double *__restrict__ q, double *__restrict__ x,
                                double *__restrict__ r, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int g = seg[i];
  if (!act[g]) return;
  const double alpha = sc[g * kScal] / sc[g * kScal + 1];
  x[i] = fma(alpha, p[i], x[i]);
  r[i] = fma(-alpha, q[i], r[i]);
}

__global__ void k_seg_update_p(const double *__restrict__ sc, const int *__restrict__ act,
                               const int32_t *__restrict__ seg, const double *__restrict__ z,
                               double *__restrict__ p, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int g = seg[i];
  if (!act[g]) return;
  p[i] = fma(sc[g * kScal + 3] / sc[g * kScal], p[i], z[i]);
}

__global__ void k_seg_shift(double *sc, int nseg) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < nseg) sc[g * kScal] = sc[g * kScal + 3];
}

}  // namespace

// second half of a segmented iteration: z = M^-1 r, rz_new, p = z + beta p
static void seg_precond_half(geneo_ctx *c, cudaStream_t s) {
  const int64_t n = c->topo.ndofs();
  const int nseg = (int)c->seg_off.size() - 1;
  double *sc = c->seg_sc.p;
  precondition(c, c->p_r.p, c->p_z.p, s, 1);
  c->launches += 3;
  k_seg_dot<<<nseg, 256, 0, s>>>(c->p_r.p, c->p_z.p, c->d_seg_off.p, sc + 3);
  k_seg_update_p<<<grid_for(n, 256), 256, 0, s>>>(sc, c->seg_act.p, c->d_seg_of.p, c->p_z.p,
                                                  c->p_p.p, n);
  k_seg_shift<<<grid_for(nseg, 256), 256, 0, s>>>(sc, nseg);
  GENEO_CHECK_LAUNCH();
}

// first half: q = A p, alpha per component, x/r update, (r, r), scalars to
// the pinned host mirror
static void seg_step_half(geneo_ctx *c, double *x, cudaStream_t s) {
  const int64_t n = c->topo.ndofs();
  const int nseg = (int)c->seg_off.size() - 1;
  double *sc = c->seg_sc.p;
  spmv(c, c->p_p.p, c->p_q.p, s, 1);
  c->launches += 3;
  k_seg_dot<<<nseg, 256, 0, s>>>(c->p_p.p, c->p_q.p, c->d_seg_off.p, sc + 1);
  k_seg_update_xr<<<grid_for(n, 256), 256, 0, s>>>(sc, c->seg_act.p, c->d_seg_of.p, c->p_p.p,
                                                   c->p_q.p, x, c->p_r.p, n);
  k_seg_dot<<<nseg, 256, 0, s>>>(c->p_r.p, c->p_r.p, c->d_seg_off.p, sc + 2);
  GENEO_CHECK_LAUNCH();
  GENEO_CUDA(cudaMemcpyAsync(c->h_seg, sc, sizeof(double) * kScal * nseg, cudaMemcpyDeviceToHost, s));
}

// [second half ; first half] of a segmented iteration on x = p_x, captured
// once per local precision, profiling switch and form
static void ensure_seg_graph(geneo_ctx *c) {
  const int cfg = ((c->loc.symv_cfg[0] * 8 + c->loc.symv_cfg[1]) * 2 + (c->grad32 ? 1 : 0)) * 2 +
                  (c->mf_persist ? 1 : 0);
  const int key = ((c->local_prec * 2 + (c->prof ? 1 : 0)) * 2 + (c->balanced ? 1 : 0)) * 256 + cfg;
  if (c->seg_exec && c->seg_key == key) return;
  if (c->seg_exec) cudaGraphExecDestroy(c->seg_exec);
  c->seg_exec = nullptr;
  c->seg_key = -1;
  const int64_t l0 = c->launches;
  const size_t nl = c->ev_local.size(), nc = c->ev_coarse.size();
  cudaStream_t cs = c->cap_stream;
  GENEO_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaGraph_t graph = nullptr;
  try {
    seg_precond_half(c, cs);
    seg_step_half(c, c->p_x.p, cs);
  } catch (...) {
    cudaStreamEndCapture(cs, &graph);
    if (graph) cudaGraphDestroy(graph);
    c->launches = l0;
    throw;
  }
  GENEO_CUDA(cudaStreamEndCapture(cs, &graph));
  cudaGraphExec_t exec = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  GENEO_CUDA(e);
  c->seg_exec = exec;
  c->seg_key = key;
  c->seg_graph_launches = c->launches - l0;
  c->launches = l0;
  // the event pairs recorded inside belong to the graph; they are not timed
  for (size_t q = nl; q < c->ev_local.size(); ++q)
    c->ev_free.insert(c->ev_free.end(), {c->ev_local[q].first, c->ev_local[q].second});
  for (size_t q = nc; q < c->ev_coarse.size(); ++q)
    c->ev_free.insert(c->ev_free.end(), {c->ev_coarse[q].first, c->ev_coarse[q].second});
  c->ev_local.resize(nl);
  c->ev_coarse.resize(nc);
}

int pcg_segments(geneo_ctx *c, const double *b, double *x, double tol, int maxit,
                 geneo_solve_info *info, cudaStream_t s) {
  if (!c->seg_ok)
    throw Error(GENEO_ERR_STATE,
                "the independent components are not contiguous in the unknown numbering "
                "(stack the problems along z)");
  const auto t0 = std::chrono::steady_clock::now();
  reserve_rhs(c, 1);
  const int64_t n = c->topo.ndofs();
  const int nseg = (int)c->seg_off.size() - 1;
  if (c->seg_sc.n < (int64_t)kScal * nseg) {
    if (c->seg_exec) cudaGraphExecDestroy(c->seg_exec);
    c->seg_exec = nullptr;
    c->seg_sc.alloc((int64_t)kScal * nseg);
    c->seg_act.alloc(nseg);
    if (c->h_seg) GENEO_CUDA(cudaFreeHost(c->h_seg));
    c->h_seg = nullptr;
    GENEO_CUDA(cudaMallocHost((void **)&c->h_seg, sizeof(double) * kScal * nseg));
  }
  c->seg_sc.zero(s);
  c->seg_ha.assign(nseg, 0);
  double *sc = c->seg_sc.p;
  const double *hs = c->h_seg;
  const int64_t *off = c->d_seg_off.p;
  const unsigned g = grid_for(n, 256);
  // with the graph, the iterations run on the context's own x (p_x)
  const bool graph = c->opt.use_graph != 0 && c->prof == false;
  double *xw = graph ? c->p_x.p : x;
  pcg_start(c, b, xw, s, 1);
  c->launches += 4;
  k_seg_dot<<<nseg, 256, 0, s>>>(b, b, off, sc + 4);
  precondition(c, c->p_r.p, c->p_z.p, s, 1);
  k_copy<<<g, 256, 0, s>>>(c->p_z.p, c->p_p.p, n);
  k_seg_dot<<<nseg, 256, 0, s>>>(c->p_r.p, c->p_z.p, off, sc + 0);
  GENEO_CHECK_LAUNCH();
  GENEO_CUDA(cudaMemcpyAsync(c->h_seg, sc, sizeof(double) * kScal * nseg, cudaMemcpyDeviceToHost, s));
  GENEO_CUDA(cudaStreamSynchronize(s));
  std::vector<double> bnorm(nseg), rel(nseg, 1.0);
  std::vector<int> st(nseg, GENEO_NOT_CONVERGED), its(nseg, 0);
  int nact = 0;
  for (int j = 0; j < nseg; ++j) {
    bnorm[j] = std::sqrt(hs[(size_t)j * kScal + 4]);
    c->seg_ha[j] = bnorm[j] > 0.0;
    if (!c->seg_ha[j]) {
      st[j] = GENEO_OK;
      rel[j] = 0.0;
    }
    nact += c->seg_ha[j];
  }
  GENEO_CUDA(cudaMemcpyAsync(c->seg_act.p, c->seg_ha.data(), sizeof(int) * nseg,
                             cudaMemcpyHostToDevice, s));
  for (int it = 1; it <= maxit && nact > 0; ++it) {
    if (it == 1) {
      seg_step_half(c, xw, s);
    } else if (graph) {
      ensure_seg_graph(c);
      GENEO_CUDA(cudaGraphLaunch(c->seg_exec, s));
      c->launches += c->seg_graph_launches;
    } else {
      seg_precond_half(c, s);
      seg_step_half(c, xw, s);
    }
    GENEO_CUDA(cudaStreamSynchronize(s));
    bool changed = false;
    for (int j = 0; j < nseg; ++j) {
      if (!c->seg_ha[j]) continue;
      its[j] = it;
      const double *h = hs + (size_t)j * kScal;
      if (!(h[1] > 0.0) || !std::isfinite(h[1]) || !std::isfinite(h[2])) {
        st[j] = GENEO_ERR_BREAKDOWN;
      } else {
        rel[j] = std::sqrt(h[2]) / bnorm[j];
        if (rel[j] <= tol) st[j] = GENEO_OK;
      }
      if (st[j] != GENEO_NOT_CONVERGED) {
        c->seg_ha[j] = 0;
        --nact;
        changed = true;
      }
    }
    if (changed && nact > 0) {
      GENEO_CUDA(cudaMemcpyAsync(c->seg_act.p, c->seg_ha.data(), sizeof(int) * nseg,
                                 cudaMemcpyHostToDevice, s));
      GENEO_CUDA(cudaStreamSynchronize(s));  // the host mask may change again next iteration
    }
  }
  if (xw != x) {
    c->launches += 1;
    k_copy<<<g, 256, 0, s>>>(xw, x, n);
    GENEO_CHECK_LAUNCH();
  }
  GENEO_CUDA(cudaStreamSynchronize(s));
  check_device_error(c, s);
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int status = GENEO_OK;
  for (int j = 0; j < nseg; ++j) {
    if (info) {
      info[j].iters = its[j];
      info[j].relres = rel[j];
      info[j].seconds = secs;
    }
    if (st[j] == GENEO_ERR_BREAKDOWN) status = GENEO_ERR_BREAKDOWN;
    else if (st[j] == GENEO_NOT_CONVERGED && status == GENEO_OK) status = GENEO_NOT_CONVERGED;
  }
  return status;
}

// ---------------------------------------------------------------------------
// Iterative refinement with accurate residuals.  In float64, b - A x cannot
// be evaluated below u ||A|| ||x|| (the gradient part of x grows like
// 1/gamma), so PCG iterates stop improving at a forward error far above the
// recurrence residual.  Each refinement step evaluates r = b - A x with the
// twice-the-working-precision residual kernel, solves A d = r with the same
// PCG and adds d to x.

int pcg_refined(geneo_ctx *c, const double *b, double *x, double tol, int maxit, int nref,
                geneo_solve_info *info, cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t n = c->topo.ndofs();
  geneo_solve_info one{};
  int status = pcg(c, b, x, tol, maxit, &one, s);
  int iters = one.iters;
  if (c->ref_r.n < n) {
    c->ref_r.alloc(n);
    c->ref_d.alloc(n);
  }
  for (int q = 0; q < nref && status >= 0; ++q) {
    c->launches += 1;
    k_residual_dd<<<grid_for(n * 8, 256), 256, 0, s>>>(c->d_rowptr.p, c->d_col.p, c->d_val.p, x,
                                                       b, c->ref_r.p, n);
    GENEO_CHECK_LAUNCH();
    const int st = pcg(c, c->ref_r.p, c->ref_d.p, tol, maxit, &one, s);
    iters += one.iters;
    if (st < 0) {
      status = st;
      break;
    }
    if (st == GENEO_NOT_CONVERGED) status = st;
    c->launches += 1;
    k_axpy1<<<grid_for(n, 256), 256, 0, s>>>(c->ref_d.p, x, n);
    GENEO_CHECK_LAUNCH();
  }
  // accurate relative residual of the returned x
  c->launches += 1;
  k_residual_dd<<<grid_for(n * 8, 256), 256, 0, s>>>(c->d_rowptr.p, c->d_col.p, c->d_val.p, x, b,
                                                     c->ref_r.p, n);
  GENEO_CHECK_LAUNCH();
  dot(c, c->ref_r.p, c->ref_r.p, n, c->scal.p + 5, s);
  dot(c, b, b, n, c->scal.p + 6, s);
  double h[2];
  GENEO_CUDA(cudaMemcpyAsync(h, c->scal.p + 5, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
  GENEO_CUDA(cudaStreamSynchronize(s));
  if (info) {
    info->iters = iters;
    info->relres = h[1] > 0 ? std::sqrt(h[0] / h[1]) : 0.0;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return status;
}

}  // namespace geneo
