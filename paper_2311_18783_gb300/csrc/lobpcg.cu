// GenEO eigenvectors: the filtered generalised eigenproblem of every
// subdomain (Sec. 3.2, GEVP "tauthresholdAS", eq. "eigAtildeBAS")
//
//   (I - xi_j^T) D_j A_j D_j (I - xi_j) V = lambda A_j^Neu V,
//   xi_j = G_j S_j^-1 G_j^T A_j,  S_j = G_j^T A_j G_j   (Sec. 2, eq. "inverseBw"),
//
// solved for every eigenvalue above the threshold by a batched LOBPCG that
// runs all subdomains in lockstep.  Each coarse vector added is
// R_j^T D_j (I - xi_j) V_jk (eq. "eigAtildeBAS" and the definition of
// V_GenEO below it).
//
// Iteration (per subdomain, float64): B-orthonormal search basis S = [X W P]
// (W = T R with T = A_j^-1 the explicit local inverse, R the block residual;
// W and P are B-orthogonalised against the locked vectors Q and X and then
// B-orthonormalised by Cholesky QR with column dropping), Rayleigh-Ritz on
// S^T L S by cyclic Jacobi, top-k Ritz pairs kept.  A Ritz pair is converged
// when ||L x - theta B x|| <= tol * max(theta, tau) ||B x||.  Converged
// leading pairs above tau are locked; a subdomain is done once a converged
// Ritz value at or below tau shows up (Ritz values increase towards the
// eigenvalues, so nothing above tau is left) or the iteration limit is hit.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <numeric>

#include "setup.hpp"
#include "small_eig.hpp"
#include "xi.hpp"

namespace geneo {

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// X[c][p] uniform in [-1, 1] on valid local rows, 0 on padding
__global__ void k_rand_block(double *X, int k, int64_t vlen, const int32_t *l2g, uint64_t seed,
                             uint64_t round) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= vlen) return;
  const bool valid = l2g[p] >= 0;
  for (int c = 0; c < k; ++c) {
    const uint64_t h = splitmix64(seed ^ splitmix64((uint64_t)p * 131 + (uint64_t)c * 7919 +
                                                     round * 104729));
    const double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);
    X[(int64_t)c * vlen + p] = valid ? 2.0 * u - 1.0 : 0.0;
  }
}

// y = M x for k columns with the local CSR of every subdomain (M = A_j or
// A_j^Neu); one thread per (local row, column)
__global__ void k_local_csr(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ lcol,
                            const double *__restrict__ val, const int32_t *__restrict__ slot_sub,
                            const int64_t *__restrict__ Noff, const int64_t *__restrict__ voff,
                            int64_t nslots, int k, int64_t vlen, const double *__restrict__ x,
                            double *__restrict__ y) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nslots * k) return;
  const int64_t slot = q % nslots;
  const int c = (int)(q / nslots);
  const int m = slot_sub[slot];
  const int64_t base = voff[m] + (int64_t)c * vlen;
  double s = 0;
  for (int64_t e = rowptr[slot]; e < rowptr[slot + 1]; ++e) s = fma(val[e], x[base + lcol[e]], s);
  y[base + (slot - Noff[m])] = s;
}

// u = G^T t (per kept vertex: signed sum over its local star)
__global__ void k_gt(const int64_t *__restrict__ sptr, const int32_t *__restrict__ srow,
                     const int8_t *__restrict__ ssgn, const int32_t *__restrict__ vslot_sub,
                     const int64_t *__restrict__ xvoff, const int64_t *__restrict__ voff,
                     const int64_t *__restrict__ voffS, int64_t nv, int k, int64_t vlen,
                     int64_t vlenS, const double *__restrict__ t, double *__restrict__ u) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nv * k) return;
  const int64_t v = q % nv;
  const int c = (int)(q / nv);
  const int m = vslot_sub[v];
  const int64_t tb = voff[m] + (int64_t)c * vlen;
  double s = 0;
  for (int64_t e = sptr[v]; e < sptr[v + 1]; ++e) s += ssgn[e] * t[tb + srow[e]];
  u[voffS[m] + (v - xvoff[m]) + (int64_t)c * vlenS] = s;
}

// u = G^T M x through the column-tetrahedron lists of the local gradient
// columns (M = A_j with every tetrahedron touching N_j, or A_j^Neu with the
// tetrahedra of Omega_j): per tetrahedron the curl of x and gamma eps M_T x
// enter, so gradients cancel inside each element instead of in assembled sums
__global__ void k_gtA_curl(const int64_t *__restrict__ ctp, const int32_t *__restrict__ ctt,
                           const double *__restrict__ ct, const int32_t *__restrict__ lidx,
                           const double *__restrict__ tcurl, const double *__restrict__ tmass,
                           const int32_t *__restrict__ col_sub, const int64_t *__restrict__ col_out,
                           const int64_t *__restrict__ voff, int64_t ncols, int k, int64_t vlen,
                           int64_t vlenS, const double *__restrict__ x, double *__restrict__ u) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= ncols * k) return;
  const int64_t a = q % ncols;
  const int c = (int)(q / ncols);
  const double *xb = x + (int64_t)c * vlen + voff[col_sub[a]];
  double s = 0;
  for (int64_t e = ctp[a]; e < ctp[a + 1]; ++e) {
    const int64_t T = ctt[e];
    const double *E = ct + e * 15;
    const int32_t *li = lidx + e * 6;
    double xv[6];
    for (int r = 0; r < 6; ++r) xv[r] = li[r] >= 0 ? xb[li[r]] : 0.0;
    double cx[3] = {0, 0, 0};
    for (int r = 0; r < 6; ++r)
      for (int d = 0; d < 3; ++d) cx[d] = fma(xv[r], tcurl[T * 18 + r * 3 + d], cx[d]);
    double v = E[0] * cx[0] + E[1] * cx[1] + E[2] * cx[2];
    for (int r = 0; r < 6; ++r) {
      if (E[3 + r] == 0.0) continue;
      double mx = 0;
      for (int f = 0; f < 6; ++f) mx = fma(tmass[T * 36 + r * 6 + f], xv[f], mx);
      v = fma(E[3 + r], mx, v);
    }
    s += v;
  }
  u[(int64_t)c * vlenS + col_out[a]] = s;
}

// out = x - A_j G w for every local row (the transpose part of xi_j), element
// by element: on tetrahedron T, A_T applied to the restriction of the
// gradient of w (w given on the kept vertices) to N_j.  The curl of a full
// element gradient vanishes, so only the edges of T outside N_j contribute a
// curl: c_T = -sum_{f notin N_j} (grad w)_f curl_f.  Row entries: tetrahedron,
// the row's local edge in it, local indices of its six edges (-1 outside N_j)
// and of its four vertices among the kept ones (-1 otherwise).
__constant__ int c_lep[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
__global__ void k_agw(const int64_t *__restrict__ rptr, const int32_t *__restrict__ rtet,
                      const int8_t *__restrict__ rpos, const int32_t *__restrict__ rlidx,
                      const int32_t *__restrict__ rvidx, const double *__restrict__ tcurl,
                      const double *__restrict__ tmass, const int32_t *__restrict__ slot_sub,
                      const int64_t *__restrict__ Noff, const int64_t *__restrict__ voff,
                      const int64_t *__restrict__ voffS, int64_t nslots, int k, int64_t vlen,
                      int64_t vlenS, const double *__restrict__ w, const double *__restrict__ y,
                      double *__restrict__ out) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nslots * k) return;
  const int64_t slot = q % nslots;
  const int c = (int)(q / nslots);
  const int m = slot_sub[slot];
  const double *wb = w + (int64_t)c * vlenS + voffS[m];
  double s = 0;
  for (int64_t e = rptr[slot]; e < rptr[slot + 1]; ++e) {
    const int64_t T = rtet[e];
    const int pe = rpos[e];
    const int32_t *li = rlidx + e * 6, *vi = rvidx + e * 4;
    double wv[4];
    for (int r = 0; r < 4; ++r) wv[r] = vi[r] >= 0 ? wb[vi[r]] : 0.0;
    double cT[3] = {0, 0, 0}, gm = 0;
    for (int f = 0; f < 6; ++f) {
      const double gf = wv[c_lep[f][1]] - wv[c_lep[f][0]];
      if (li[f] < 0) {
        for (int d = 0; d < 3; ++d) cT[d] = fma(-gf, tcurl[T * 18 + f * 3 + d], cT[d]);
      } else {
        gm = fma(tmass[T * 36 + pe * 6 + f], gf, gm);
      }
    }
    s += tcurl[T * 18 + pe * 3 + 0] * cT[0] + tcurl[T * 18 + pe * 3 + 1] * cT[1] +
         tcurl[T * 18 + pe * 3 + 2] * cT[2] + gm;
  }
  const int64_t p = voff[m] + (slot - Noff[m]) + (int64_t)c * vlen;
  out[p] = y[p] - s;
}

// out = x - G u (mode 1) or out = G u (mode 0), per local row
__global__ void k_g(const int32_t *__restrict__ ghead, const int32_t *__restrict__ gtail,
                    const int32_t *__restrict__ slot_sub, const int64_t *__restrict__ Noff,
                    const int64_t *__restrict__ voff, const int64_t *__restrict__ voffS,
                    int64_t nslots, int k, int64_t vlen, int64_t vlenS,
                    const double *__restrict__ u, const double *__restrict__ x,
                    double *__restrict__ out, int mode, const double *__restrict__ scale) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nslots * k) return;
  const int64_t slot = q % nslots;
  const int c = (int)(q / nslots);
  const int m = slot_sub[slot];
  const int64_t ub = voffS[m] + (int64_t)c * vlenS;
  double g = 0;
  if (ghead[slot] >= 0) g += u[ub + ghead[slot]];
  if (gtail[slot] >= 0) g -= u[ub + gtail[slot]];
  const int64_t p = voff[m] + (slot - Noff[m]) + (int64_t)c * vlen;
  if (mode == 2) out[p] += scale ? scale[m] * g : g;
  else out[p] = mode ? x[p] - g : g;
}

// float32 part of the split local inverse (Sec. 2, eq. "inverseBw"):
// C_j = A_j^-1 - G_j S_j^-1 G_j^T = (I - xi_j) A_j^-1, formed in float64 from
// the explicit inverse and S_j^-1 and stored in float32 (padding: identity)
__device__ __forceinline__ double sinv_at(const double *sinv, int64_t toffS, int v, int w) {
  if (v < w) {
    const int t = v;
    v = w;
    w = t;
  }
  const int I = v / kTile, J = w / kTile;
  return sinv[(toffS + (int64_t)I * (I + 1) / 2 + J) * kTileElems + (v % kTile) * kTile + (w % kTile)];
}

__global__ void k_split_cast(const double *__restrict__ ainv, const int32_t *__restrict__ nt,
                             const int64_t *__restrict__ toff, const int64_t *__restrict__ Noff,
                             const int32_t *__restrict__ ghead, const int32_t *__restrict__ gtail,
                             const double *__restrict__ sinv, const int64_t *__restrict__ toffS,
                             const double *__restrict__ gfac, float *__restrict__ out) {
  const int m = blockIdx.y;
  const int64_t ntm = nt[m];
  const int64_t q = blockIdx.x;
  if (q >= ntm * (ntm + 1) / 2) return;
  int I = (int)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
  while ((int64_t)(I + 1) * (I + 2) / 2 <= q) ++I;
  while ((int64_t)I * (I + 1) / 2 > q) --I;
  const int J = (int)(q - (int64_t)I * (I + 1) / 2);
  const int64_t ni = Noff[m + 1] - Noff[m];
  const int64_t tb = (toff[m] + q) * kTileElems;
  for (int e = threadIdx.x; e < kTileElems; e += blockDim.x) {
    const int64_t r = (int64_t)I * kTile + (e >> 6), cc = (int64_t)J * kTile + (e & 63);
    double v = ainv[tb + e];
    if (r < ni && cc < ni) {
      const int64_t sr = Noff[m] + r, sc = Noff[m] + cc;
      const int hr = ghead[sr], tr = gtail[sr], hc = ghead[sc], tc = gtail[sc];
      double g = 0;
      if (hr >= 0 && hc >= 0) g += sinv_at(sinv, toffS[m], hr, hc);
      if (hr >= 0 && tc >= 0) g -= sinv_at(sinv, toffS[m], hr, tc);
      if (tr >= 0 && hc >= 0) g -= sinv_at(sinv, toffS[m], tr, hc);
      if (tr >= 0 && tc >= 0) g += sinv_at(sinv, toffS[m], tr, tc);
      v -= gfac ? gfac[m] * g : g;
    }
    out[tb + e] = (float)v;
  }
}

__global__ void k_take(const double *__restrict__ src, const int32_t *__restrict__ idx,
                       double *__restrict__ dst, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

__global__ void k_gather_sum_i64(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                 const double *__restrict__ src, int64_t n,
                                 double *__restrict__ out) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  double s = 0;
  for (int64_t k = ptr[r]; k < ptr[r + 1]; ++k) s += src[idx[k]];
  out[r] = s;
}

// y = d .* x on k columns
__global__ void k_dscale(const double *__restrict__ d, int k, int64_t vlen,
                         const double *__restrict__ x, double *__restrict__ y) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= vlen) return;
  const double dv = d[p];
  for (int c = 0; c < k; ++c) y[(int64_t)c * vlen + p] = dv * x[(int64_t)c * vlen + p];
}

// y = a - b on n elements
__global__ void k_sub(const double *__restrict__ a, const double *__restrict__ b,
                      double *__restrict__ y, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = a[i] - b[i];
}

// One-pass Gram blocks: CTA (m, chunk, sub-block) reads rows of subdomain
// m's segment once and accumulates an 8 x 8 block of <X_a, Y_b> in
// registers; the per-chunk partials are summed in chunk order by
// k_gram_final (deterministic).  part[(m * nch + chunk) * 256 + a * 16 + b].
constexpr int kGramChunks = 4;
__global__ void __launch_bounds__(256)
    k_gram_part(const double *__restrict__ X, int ka, const double *__restrict__ Y, int kb,
                int64_t vlen, const int64_t *__restrict__ voff, double *__restrict__ part) {
  const int m = blockIdx.x, ch = blockIdx.y;
  const int a0 = (blockIdx.z >> 1) * 8, b0 = (blockIdx.z & 1) * 8;
  const int na = min(8, ka - a0), nb = min(8, kb - b0);
  if (na <= 0 || nb <= 0) return;
  const int64_t s0 = voff[m], s1 = voff[m + 1];
  const int64_t len = s1 - s0, per = (len + kGramChunks - 1) / kGramChunks;
  const int64_t c0 = s0 + ch * per, c1 = min(s1, c0 + per);
  double acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0;
  for (int64_t p = c0 + threadIdx.x; p < c1; p += blockDim.x) {
    double xv[8], yv[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) xv[i] = i < na ? X[(int64_t)(a0 + i) * vlen + p] : 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) yv[j] = j < nb ? Y[(int64_t)(b0 + j) * vlen + p] : 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = fma(xv[i], yv[j], acc[i][j]);
  }
  __shared__ double sh[8][64];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      double v = acc[i][j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (l == 0) sh[w][i * 8 + j] = v;
    }
  __syncthreads();
  if (threadIdx.x < 64) {
    const int i = threadIdx.x >> 3, j = threadIdx.x & 7;
    double v = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += sh[q][threadIdx.x];
    part[((int64_t)m * kGramChunks + ch) * 256 + (a0 + i) * 16 + (b0 + j)] = v;
  }
}

__global__ void k_gram_final(const double *__restrict__ part, int ka, int kb, int ldg,
                             double *__restrict__ G) {
  const int m = blockIdx.x, e = threadIdx.x;
  const int a = e >> 4, b = e & 15;
  if (a >= ka || b >= kb) return;
  double v = 0;
  for (int ch = 0; ch < kGramChunks; ++ch) v += part[((int64_t)m * kGramChunks + ch) * 256 + e];
  G[((int64_t)m * ldg + a) * ldg + b] = v;
}

// out[c] = sum_j src_j * C[m][j][c] over nsrc source columns given by
// pointers (column-major blocks of length vlen); one thread per position
struct SrcList {
  const double *p[96];
};
__global__ void k_combine(SrcList src, int nsrc, const double *__restrict__ C, int ldc, int kout,
                          const int32_t *__restrict__ pos_sub, int64_t vlen,
                          double *__restrict__ out) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= vlen) return;
  const int m = pos_sub[p];
  const double *Cm = C + (int64_t)m * ldc * ldc;
  double sv[96];
  for (int j = 0; j < nsrc; ++j) sv[j] = src.p[j][p];
  for (int c = 0; c < kout; ++c) {
    double s = 0;
    for (int j = 0; j < nsrc; ++j) s = fma(sv[j], Cm[j * ldc + c], s);
    out[(int64_t)c * vlen + p] = s;
  }
}

// copy column cs of block X into column cd of block Q for the subdomains
// listed with a flag
__global__ void k_copy_cols(const double *__restrict__ X, double *__restrict__ Q,
                            const int32_t *__restrict__ pos_sub, const int32_t *__restrict__ src_col,
                            const int32_t *__restrict__ dst_col, int nmoves_per_sub, int64_t vlen) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= vlen) return;
  const int m = pos_sub[p];
  for (int t = 0; t < nmoves_per_sub; ++t) {
    const int s = src_col[m * nmoves_per_sub + t];
    const int d = dst_col[m * nmoves_per_sub + t];
    if (s < 0 || d < 0) continue;
    Q[(int64_t)d * vlen + p] = X[(int64_t)s * vlen + p];
  }
}

// ---- per-subdomain small dense kernels (one thread per subdomain) ----------

// Cholesky of the Gram matrix G (n x n at ld) with column dropping; writes
// T = R^-1 (upper, so Y T is orthonormal) into Tout, dropped columns zero.
__global__ void k_cholqr_factor(const double *__restrict__ Gall, int n, int ld,
                                double *__restrict__ Tall, int nsub) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nsub) return;
  const double *G = Gall + (int64_t)m * ld * ld;
  double *T = Tall + (int64_t)m * ld * ld;
  double R[96 * 97 / 2 + 96];
  auto r = [&](int i, int j) -> double & { return R[j * (j + 1) / 2 + i]; };  // i <= j
  bool keep[96];
  double gmax = 0;
  for (int i = 0; i < n; ++i) gmax = fmax(gmax, G[i * ld + i]);
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i <= j; ++i) {
      double s = G[i * ld + j];
      for (int t = 0; t < i; ++t) s -= r(t, i) * r(t, j);
      if (i < j) {
        r(i, j) = keep[i] ? s / r(i, i) : 0.0;
      } else {
        const double d = s;
        keep[j] = d > 1e-13 * gmax && d > 0.0;
        r(j, j) = keep[j] ? sqrt(d) : 1.0;
      }
    }
    if (!keep[j])
      for (int i = 0; i < j; ++i) r(i, j) = 0.0;
  }
  // T = R^-1 (upper triangular), zero columns for dropped ones
  for (int i = 0; i < n * ld; ++i) T[i] = 0.0;
  for (int c = 0; c < n; ++c) {
    if (!keep[c]) continue;
    // solve R t = e_c for the column c of T (back substitution)
    for (int i = c; i >= 0; --i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int t = i + 1; t <= c; ++t) s -= r(i, t) * T[t * ld + c];
      T[i * ld + c] = keep[i] ? s / r(i, i) : 0.0;
    }
  }
}

// Symmetric eigen-decomposition of the n x n matrix H (at ld) by cyclic
// Jacobi; writes the top kout eigenvalues (descending) and eigenvectors
// (columns of V, n x kout at ld).
__global__ void k_rr_jacobi(const double *__restrict__ Hall, int n, int ld, int kout,
                            double *__restrict__ theta, double *__restrict__ Vall, int nsub) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nsub) return;
  const double *Hg = Hall + (int64_t)m * ld * ld;
  double *Vo = Vall + (int64_t)m * ld * ld;
  double a[48 * 48], v[48 * 48];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      a[i * n + j] = 0.5 * (Hg[i * ld + j] + Hg[j * ld + i]);
      v[i * n + j] = (i == j) ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0, tot = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += a[i * n + j] * a[i * n + j];
        if (i != j) off += a[i * n + j] * a[i * n + j];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[p * n + q];
        if (fabs(apq) < 1e-300) continue;
        const double app = a[p * n + p], aqq = a[q * n + q];
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int k2 = 0; k2 < n; ++k2) {
          const double akp = a[k2 * n + p], akq = a[k2 * n + q];
          a[k2 * n + p] = c * akp - s * akq;
          a[k2 * n + q] = s * akp + c * akq;
        }
        for (int k2 = 0; k2 < n; ++k2) {
          const double apk = a[p * n + k2], aqk = a[q * n + k2];
          a[p * n + k2] = c * apk - s * aqk;
          a[q * n + k2] = s * apk + c * aqk;
        }
        for (int k2 = 0; k2 < n; ++k2) {
          const double vkp = v[k2 * n + p], vkq = v[k2 * n + q];
          v[k2 * n + p] = c * vkp - s * vkq;
          v[k2 * n + q] = s * vkp + c * vkq;
        }
      }
  }
  int idx[48];
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (a[idx[j] * n + idx[j]] > a[idx[i] * n + idx[i]]) {
        const int t = idx[i];
        idx[i] = idx[j];
        idx[j] = t;
      }
  for (int c = 0; c < kout; ++c) {
    theta[m * kout + c] = a[idx[c] * n + idx[c]];
    for (int i = 0; i < n; ++i) Vo[i * ld + c] = v[i * n + idx[c]];
    for (int i = n; i < ld; ++i) Vo[i * ld + c] = 0.0;
  }
}

// The same eigen-decomposition with one CTA per subdomain: parallel cyclic
// Jacobi (Brent and Luk's ordering: each sweep is n - 1 rounds of n / 2
// disjoint index pairs from the round-robin tournament, all rotations of a
// round computed from the same matrix and applied together), with the
// matrix and the rotations accumulated in shared memory.  n <= 48.
constexpr int kJacMax = 48;
__global__ void __launch_bounds__(256)
    k_rr_jacobi_cta(const double *__restrict__ Hall, int n, int ld, int kout,
                    double *__restrict__ theta, double *__restrict__ Vall) {
  __shared__ double a[kJacMax][kJacMax + 1], v[kJacMax][kJacMax + 1];
  __shared__ double cs[kJacMax / 2], sn[kJacMax / 2], red[256 / 32][2];
  __shared__ int pp[kJacMax / 2], qq[kJacMax / 2], idx[kJacMax];
  __shared__ int stop;
  const int m = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const double *Hg = Hall + (int64_t)m * ld * ld;
  double *Vo = Vall + (int64_t)m * ld * ld;
  // an odd n gets one idle index (its pairs are skipped)
  const int ne = n + (n & 1), np = ne / 2;
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e % n;
    a[i][j] = 0.5 * (Hg[i * ld + j] + Hg[j * ld + i]);
    v[i][j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 30; ++sweep) {
    // convergence test: off-diagonal mass against the total
    double off = 0, tot = 0;
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, j = e % n;
      const double x = a[i][j] * a[i][j];
      tot += x;
      if (i != j) off += x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if ((tid & 31) == 0) {
      red[tid >> 5][0] = off;
      red[tid >> 5][1] = tot;
    }
    __syncthreads();
    if (tid == 0) {
      double so = 0, st = 0;
      for (int w = 0; w < (nt >> 5); ++w) {
        so += red[w][0];
        st += red[w][1];
      }
      stop = so <= 1e-30 * st;
    }
    __syncthreads();
    if (stop) break;
    for (int r = 0; r < ne - 1; ++r) {
      // pairs of round r and their rotations
      if (tid < np) {
        int p, q;
        if (tid == 0) {
          p = r;
          q = ne - 1;
        } else {
          p = (r + tid) % (ne - 1);
          q = (r - tid + ne - 1) % (ne - 1);
        }
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, sv = 0.0;
        if (q < n) {
          const double apq = a[p][q];
          if (fabs(apq) >= 1e-300) {
            const double tau = (a[q][q] - a[p][p]) / (2.0 * apq);
            const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sv = t * c;
          }
        }
        pp[tid] = p;
        qq[tid] = q < n ? q : p;  // an idle pair rotates nothing
        cs[tid] = c;
        sn[tid] = q < n ? sv : 0.0;
      }
      __syncthreads();
      // columns: A <- A J ; V <- V J
      for (int e = tid; e < np * n; e += nt) {
        const int k = e / n, i = e % n;
        const int p = pp[k], q = qq[k];
        if (p == q) continue;
        const double c = cs[k], sv = sn[k];
        const double aip = a[i][p], aiq = a[i][q];
        a[i][p] = c * aip - sv * aiq;
        a[i][q] = sv * aip + c * aiq;
        const double vip = v[i][p], viq = v[i][q];
        v[i][p] = c * vip - sv * viq;
        v[i][q] = sv * vip + c * viq;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = tid; e < np * n; e += nt) {
        const int k = e / n, j = e % n;
        const int p = pp[k], q = qq[k];
        if (p == q) continue;
        const double c = cs[k], sv = sn[k];
        const double apj = a[p][j], aqj = a[q][j];
        a[p][j] = c * apj - sv * aqj;
        a[q][j] = sv * apj + c * aqj;
      }
      __syncthreads();
    }
  }
  // descending order of the diagonal (ties keep the lower index first)
  if (tid < n) {
    const double d = a[tid][tid];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double e = a[j][j];
      rank += (e > d) || (e == d && j < tid);
    }
    idx[rank] = tid;
  }
  __syncthreads();
  for (int e = tid; e < kout * ld; e += nt) {
    const int c = e / ld, i = e % ld;
    const int src = idx[c];
    if (i == 0) theta[m * kout + c] = a[src][src];
    Vo[i * ld + c] = i < n ? v[i][src] : 0.0;
  }
}

// R = LX - BX diag(theta); norms of R and BX per (m, c)
__global__ void k_resid(const double *__restrict__ LX, const double *__restrict__ BX,
                        const double *__restrict__ theta, int k, const int32_t *__restrict__ pos_sub,
                        int64_t vlen, double *__restrict__ R) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= vlen) return;
  const int m = pos_sub[p];
  for (int c = 0; c < k; ++c) {
    const int64_t i = (int64_t)c * vlen + p;
    R[i] = LX[i] - theta[m * k + c] * BX[i];
  }
}

// A_j^Neu values (on the local CSR of N_j) into the tile-packed layout of the
// local factors, lower tiles only, with the diagonal scaled by 1 + delta
__global__ void k_neumann_tiles(const int64_t *__restrict__ Noff, const int64_t *__restrict__ lrowptr,
                                const int32_t *__restrict__ lcol, const double *__restrict__ nval,
                                const int64_t *__restrict__ toff, double delta,
                                double *__restrict__ tiles) {
  const int m = blockIdx.y;
  const int64_t ni = Noff[m + 1] - Noff[m];
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < ni;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t slot = Noff[m] + r;
    const int I = (int)(r / kTile), rr = (int)(r % kTile);
    for (int64_t q = lrowptr[slot]; q < lrowptr[slot + 1]; ++q) {
      const int c = lcol[q];
      const int J = c / kTile;
      if (J > I) continue;
      const double v = (c == r) ? nval[q] * (1.0 + delta) : nval[q];
      tiles[(toff[m] + (int64_t)I * (I + 1) / 2 + J) * kTileElems + rr * kTile + (c % kTile)] = v;
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side

struct Lobpcg {
  geneo_ctx *c;
  cudaStream_t s;
  XiOp &op;
  int nsub, k;
  int64_t vlen;
  // blocks (k columns each)
  DevBuf<double> X, LX, BX, W, LW, BW, P, LP, BP, R, T1, T2, T3, U1, U2;
  DevBuf<double> Q, BQ;
  int qcap = 0;
  std::vector<int> nq;  // locked per subdomain
  DevBuf<double> gram, coef, theta, tmat, gpart;
  int ld = 0;
  Lobpcg(geneo_ctx *cc, cudaStream_t ss, XiOp &o) : c(cc), s(ss), op(o) {}
};

static void apply_sparse(Lobpcg &L, const DevBuf<double> &vals, const double *x, double *y, int k) {
  const int64_t tot = L.op.nslots * k;
  k_local_csr<<<grid_for(tot, 256), 256, 0, L.s>>>(L.op.lrp.p, L.op.lcol.p, vals.p, L.op.slot_sub.p, L.op.Noff.p,
                                                   L.c->loc.d_voff.p, L.op.nslots, k, L.vlen, x, y);
}

static void apply_B(Lobpcg &L, const double *Y, double *BY, int k) {
  apply_sparse(L, L.op.nval, Y, BY, k);
}

// out = x - xi x (mode 1) with xi = G S^-1 G^T A, or out = x - xi^T x =
// x - A G S^-1 G^T x (mode 2).  Uses U1, U2 as scratch.
static void xi_apply(Lobpcg &L, const double *x, double *out, int k, int mode) {
  if (mode == 1) {
    k_gtA_curl<<<grid_for(L.op.nv * k, 128), 128, 0, L.s>>>(
        L.op.ctp_d.p, L.op.ctt_d.p, L.op.ct_d.p, L.op.lidx_d.p, L.op.tcurl.p, L.op.tmass.p, L.op.col_sub.p,
        L.op.col_out.p, L.c->loc.d_voff.p, L.op.nv, k, L.vlen, L.op.vlenS, x, L.U1.p);
  } else {
    k_gt<<<grid_for(L.op.nv * k, 256), 256, 0, L.s>>>(L.op.sptr.p, L.op.srow.p, L.op.ssgn.p, L.op.vslot_sub.p,
                                                   L.op.xvoff.p, L.c->loc.d_voff.p, L.op.sb.d_voff.p,
                                                   L.op.nv, k, L.vlen, L.op.vlenS, x, L.U1.p);
  }
  for (int col = 0; col < k; ++col)
    symv_batch<double>(L.op.sb, L.op.s_inv.p, L.U1.p + (int64_t)col * L.op.vlenS,
                       L.U2.p + (int64_t)col * L.op.vlenS, L.c->d_err.p, L.s);
  if (mode == 1) {
    k_g<<<grid_for(L.op.nslots * k, 256), 256, 0, L.s>>>(L.op.ghead.p, L.op.gtail.p, L.op.slot_sub.p, L.op.Noff.p,
                                                      L.c->loc.d_voff.p, L.op.sb.d_voff.p, L.op.nslots, k,
                                                      L.vlen, L.op.vlenS, L.U2.p, x, out, 1, nullptr);
  } else {
    k_agw<<<grid_for(L.op.nslots * k, 128), 128, 0, L.s>>>(
        L.op.rptr.p, L.op.rtet.p, L.op.rpos.p, L.op.rlidx.p, L.op.rvidx.p, L.op.tcurl.p, L.op.tmass.p, L.op.slot_sub.p,
        L.op.Noff.p, L.c->loc.d_voff.p, L.op.sb.d_voff.p, L.op.nslots, k, L.vlen, L.op.vlenS, L.U2.p, x, out);
  }
}

static bool classical_pencil(const Lobpcg &L) {
  return L.c->opt.geneo_pencil == GENEO_PENCIL_CLASSICAL;
}

// Y <- Y - G S_B^-1 G^T B Y: the B-orthogonal projection away from the
// gradients, where the eigenvectors of the filtered GEVP live (for g = G c
// in the null space of L, g^T L v = 0 = lambda g^T B v).  The classical
// pencil has no such null space: no projection.
static void project_gradients_B(Lobpcg &L, double *Y, int k) {
  if (classical_pencil(L)) return;
  k_gtA_curl<<<grid_for(L.op.nv * k, 128), 128, 0, L.s>>>(
      L.op.ctp_n.p, L.op.ctt_n.p, L.op.ct_n.p, L.op.lidx_n.p, L.op.tcurl.p, L.op.tmass.p, L.op.col_sub.p, L.op.col_out.p,
      L.c->loc.d_voff.p, L.op.nv, k, L.vlen, L.op.vlenS, Y, L.U1.p);
  for (int col = 0; col < k; ++col)
    symv_batch<double>(L.op.sb, L.op.sn_inv.p, L.U1.p + (int64_t)col * L.op.vlenS,
                       L.U2.p + (int64_t)col * L.op.vlenS, L.c->d_err.p, L.s);
  k_g<<<grid_for(L.op.nslots * k, 256), 256, 0, L.s>>>(L.op.ghead.p, L.op.gtail.p, L.op.slot_sub.p, L.op.Noff.p,
                                                    L.c->loc.d_voff.p, L.op.sb.d_voff.p, L.op.nslots, k,
                                                    L.vlen, L.op.vlenS, L.U2.p, Y, Y, 1, nullptr);
}

// LY = (I - xi)^T D A D (I - xi) Y  for a block of k columns (Sec. 3.2,
// eq. "eigAtildeBAS"), or D A D Y for the classical pencil of the remark in
// Sec. 3.2 (eq. "eigGenEOClassis")
static void apply_L(Lobpcg &L, const double *Y, double *LY, int k) {
  const int64_t tot = L.vlen * k;
  if (classical_pencil(L)) {
    k_dscale<<<grid_for(L.vlen, 256), 256, 0, L.s>>>(L.op.dmask.p, k, L.vlen, Y, L.T2.p);
    apply_sparse(L, L.op.aval, L.T2.p, L.T1.p, k);         // T1 = A D Y
    k_dscale<<<grid_for(L.vlen, 256), 256, 0, L.s>>>(L.op.dmask.p, k, L.vlen, L.T1.p, LY);
    return;
  }
  xi_apply(L, Y, L.T1.p, k, 1);                        // T1 = (I - xi) Y
  k_dscale<<<grid_for(L.vlen, 256), 256, 0, L.s>>>(L.op.dmask.p, k, L.vlen, L.T1.p, L.T2.p);
  apply_sparse(L, L.op.aval, L.T2.p, L.T1.p, k);           // T1 = A D (I - xi) Y
  k_dscale<<<grid_for(L.vlen, 256), 256, 0, L.s>>>(L.op.dmask.p, k, L.vlen, L.T1.p, L.T2.p);
  xi_apply(L, L.T2.p, LY, k, 2);                       // LY = T2 - A G S^-1 G^T T2
  (void)tot;
}


static void gram(Lobpcg &L, const double *X, int ka, const double *Y, int kb, double *G) {
  if (L.gpart.n < (int64_t)L.nsub * kGramChunks * 256) L.gpart.alloc((int64_t)L.nsub * kGramChunks * 256);
  const int zb = (ka > 8 || kb > 8) ? 4 : 1;  // sub-blocks (a0, b0): z = 2 (a0 / 8) + b0 / 8
  k_gram_part<<<dim3(L.nsub, kGramChunks, zb), 256, 0, L.s>>>(X, ka, Y, kb, L.vlen,
                                                              L.c->loc.d_voff.p, L.gpart.p);
  k_gram_final<<<L.nsub, 256, 0, L.s>>>(L.gpart.p, ka, kb, L.ld, G);
}

// out (kout columns) = sum over source columns * coef[m]
static void combine(Lobpcg &L, const std::vector<const double *> &src, const double *coef,
                    int kout, double *out) {
  SrcList sl;
  for (size_t j = 0; j < src.size(); ++j) sl.p[j] = src[j];
  k_combine<<<grid_for(L.vlen, 128), 128, 0, L.s>>>(sl, (int)src.size(), coef, L.ld, kout,
                                                    L.op.pos_sub.p, L.vlen, out);
}

static std::vector<const double *> cols(const DevBuf<double> &b, int k, int64_t vlen) {
  std::vector<const double *> v;
  for (int j = 0; j < k; ++j) v.push_back(b.p + (int64_t)j * vlen);
  return v;
}

// Y <- Y - V (BV^T Y) for one block V of kv <= k columns (B-inner products)
static void project_block(Lobpcg &L, DevBuf<double> &Y, const double *V, const double *BV, int kv,
                          int k) {
  const int ld = L.ld;
  gram(L, BV, kv, Y.p, k, L.gram.p);
  std::vector<double> hg = L.gram.download(L.s);
  std::vector<double> cf((size_t)L.nsub * ld * ld, 0.0);
  for (int m = 0; m < L.nsub; ++m)
    for (int j = 0; j < k; ++j) {
      cf[(size_t)m * ld * ld + j * ld + j] = 1.0;
      if (j < kv)
        for (int cc = 0; cc < k; ++cc)
          cf[(size_t)m * ld * ld + (k + j) * ld + cc] = -hg[(size_t)m * ld * ld + j * ld + cc];
    }
  L.coef.upload(cf, L.s);
  std::vector<const double *> src = cols(Y, k, L.vlen);
  for (int j = 0; j < kv; ++j) src.push_back(V + (int64_t)j * L.vlen);
  combine(L, src, L.coef.p, k, L.T1.p);
  GENEO_CUDA(cudaMemcpyAsync(Y.p, L.T1.p, sizeof(double) * L.vlen * k, cudaMemcpyDeviceToDevice, L.s));
}

// Y <- Y - Q (BQ^T Y) - X (BX^T Y): locked vectors in chunks of k columns
// (subdomains with fewer locked vectors see zero columns), then X
static void b_orthogonalize(Lobpcg &L, DevBuf<double> &Y, const DevBuf<double> *Xb,
                            const DevBuf<double> *BXb, int kx, bool with_q, int k) {
  if (with_q) {
    int maxq = 0;
    for (int v : L.nq) maxq = std::max(maxq, v);
    for (int q0 = 0; q0 < maxq; q0 += k)
      project_block(L, Y, L.Q.p + (int64_t)q0 * L.vlen, L.BQ.p + (int64_t)q0 * L.vlen,
                    std::min(k, maxq - q0), k);
  }
  if (Xb) project_block(L, Y, Xb->p, BXb->p, kx, k);
}

// B-orthonormalise Y in place (two passes of Cholesky QR); BY (and LY if
// given) are transformed alike; BY must equal B Y on entry.
static void cholqr(Lobpcg &L, DevBuf<double> &Y, DevBuf<double> &BY, DevBuf<double> *LY, int k) {
  for (int pass = 0; pass < 2; ++pass) {
    gram(L, Y.p, k, BY.p, k, L.gram.p);
    k_cholqr_factor<<<grid_for(L.nsub, 32), 32, 0, L.s>>>(L.gram.p, k, L.ld, L.tmat.p, L.nsub);
    combine(L, cols(Y, k, L.vlen), L.tmat.p, k, L.T1.p);
    GENEO_CUDA(cudaMemcpyAsync(Y.p, L.T1.p, sizeof(double) * L.vlen * k, cudaMemcpyDeviceToDevice, L.s));
    combine(L, cols(BY, k, L.vlen), L.tmat.p, k, L.T1.p);
    GENEO_CUDA(cudaMemcpyAsync(BY.p, L.T1.p, sizeof(double) * L.vlen * k, cudaMemcpyDeviceToDevice, L.s));
    if (LY) {
      combine(L, cols(*LY, k, L.vlen), L.tmat.p, k, L.T1.p);
      GENEO_CUDA(cudaMemcpyAsync(LY->p, L.T1.p, sizeof(double) * L.vlen * k, cudaMemcpyDeviceToDevice, L.s));
    }
  }
}

static void grow_q(Lobpcg &L, int need) {
  if (need <= L.qcap) return;
  int cap = std::max(need, std::max(16, 2 * L.qcap));
  DevBuf<double> nQ, nBQ;
  nQ.alloc((int64_t)cap * L.vlen);
  nBQ.alloc((int64_t)cap * L.vlen);
  nQ.zero(L.s);
  nBQ.zero(L.s);
  if (L.qcap) {
    GENEO_CUDA(cudaMemcpyAsync(nQ.p, L.Q.p, sizeof(double) * L.vlen * L.qcap, cudaMemcpyDeviceToDevice, L.s));
    GENEO_CUDA(cudaMemcpyAsync(nBQ.p, L.BQ.p, sizeof(double) * L.vlen * L.qcap, cudaMemcpyDeviceToDevice, L.s));
  }
  GENEO_CUDA(cudaStreamSynchronize(L.s));
  std::swap(L.Q.p, nQ.p);
  std::swap(L.Q.n, nQ.n);
  std::swap(L.BQ.p, nBQ.p);
  std::swap(L.BQ.n, nBQ.n);
  L.qcap = cap;
}

__global__ void k_pos_tables(const int32_t *__restrict__ l2g, const int32_t *__restrict__ owner,
                             const int32_t *__restrict__ vrow_m, int64_t vlen,
                             int32_t *__restrict__ pos_sub, double *__restrict__ dmask) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= vlen) return;
  const int m = vrow_m[p / kTile];
  pos_sub[p] = m;
  const int32_t g = l2g[p];
  dmask[p] = (g >= 0 && owner[g] == m) ? 1.0 : 0.0;
}

// A subdomain whose edges all join boundary vertices (a thin box between a
// hole and the outer boundary) has no gradient column: its S_j is empty and
// is stored as one padded 1x1 block, which gets the unit pivot here so that
// the batched inverse stays defined (no vector entry ever reaches it).
static void unit_empty_gradient_blocks(const TileBatch &b, const LocalStructure &ls, int nsub,
                                       double *data, cudaStream_t s) {
  static const double one = 1.0;
  for (int m = 0; m < nsub; ++m)
    if (ls.xv_off[m + 1] == ls.xv_off[m])
      GENEO_CUDA(cudaMemcpyAsync(data + b.toff[m] * kTileElems, &one, sizeof(double),
                                 cudaMemcpyHostToDevice, s));
}

// local operators of every subdomain: A_j and A_j^Neu values on the local
// CSR, the Boolean D_j, the gradient structure of xi_j and the inverses of
// S_j = G_j^T A_j G_j (Galerkin per tetrahedron, tiled Cholesky inverse)
void build_xi_operator(geneo_ctx *c, XiOp &L, cudaStream_t s) {
  L.vlen = c->loc.vlen;
  const Decomposition &d = c->dec;
  const LocalStructure &ls = c->ls;
  L.nslots = d.N_off[d.nsub];
  std::vector<int32_t> slot_sub(L.nslots);
  for (int m = 0; m < d.nsub; ++m)
    for (int64_t q = d.N_off[m]; q < d.N_off[m + 1]; ++q) slot_sub[q] = m;
  L.slot_sub.upload(slot_sub, s);
  L.Noff.upload(d.N_off, s);
  L.lrp.upload(ls.lrowptr, s);
  L.lcol.upload(ls.lcol, s);
  {
    DevBuf<int32_t> lpos;
    lpos.upload(ls.lpos, s);
    L.aval.alloc(lpos.n);
    k_take<<<grid_for(lpos.n, 256), 256, 0, s>>>(c->d_val.p, lpos.p, L.aval.p, lpos.n);
    DevBuf<int64_t> ncp;
    DevBuf<int32_t> nci;
    ncp.upload(ls.ncptr, s);
    nci.upload(ls.ncidx, s);
    L.nval.alloc(lpos.n);
    k_gather_sum_i64<<<grid_for(lpos.n, 256), 256, 0, s>>>(ncp.p, nci.p, c->d_Ae.p, lpos.n, L.nval.p);
    DevBuf<int32_t> own;
    own.upload(d.owner, s);
    L.pos_sub.alloc(L.vlen);
    L.dmask.alloc(L.vlen);
    k_pos_tables<<<grid_for(L.vlen, 256), 256, 0, s>>>(c->d_l2g.p, own.p, c->loc.d_vrow_m.p, L.vlen,
                                                       L.pos_sub.p, L.dmask.p);
    GENEO_CHECK_LAUNCH();
    GENEO_CUDA(cudaStreamSynchronize(s));
  }
  L.ghead.upload(ls.gi_head, s);
  L.gtail.upload(ls.gi_tail, s);
  L.sptr.upload(ls.star_ptr, s);
  L.srow.upload(ls.star_row, s);
  L.ssgn.upload(ls.star_sgn, s);
  L.xvoff.upload(ls.xv_off, s);
  L.nv = ls.xv_off[d.nsub];
  std::vector<int32_t> vsub(L.nv);
  std::vector<int64_t> dims(d.nsub);
  for (int m = 0; m < d.nsub; ++m) {
    dims[m] = std::max<int64_t>(1, ls.xv_off[m + 1] - ls.xv_off[m]);
    for (int64_t v = ls.xv_off[m]; v < ls.xv_off[m + 1]; ++v) vsub[v] = m;
  }
  L.vslot_sub.upload(vsub, s);
  // S_j columns: the local gradient of each kept vertex, restricted to N_j
  Columns X;
  for (int m = 0; m < d.nsub; ++m)
    for (int64_t v = ls.xv_off[m]; v < ls.xv_off[m + 1]; ++v) {
      std::vector<std::pair<int32_t, double>> ent;
      for (int64_t e = ls.star_ptr[v]; e < ls.star_ptr[v + 1]; ++e)
        ent.push_back({d.N_idx[d.N_off[m] + ls.star_row[e]], (double)ls.star_sgn[e]});
      std::sort(ent.begin(), ent.end());
      for (auto &pr : ent) {
        X.row.push_back(pr.first);
        X.val.push_back(pr.second);
      }
      X.ptr.push_back((int64_t)X.row.size());
      X.mat.push_back(m);
      X.loc.push_back((int32_t)(v - ls.xv_off[m]));
    }
  L.sb.layout(dims);
  L.sb.upload_meta(s);
  L.vlenS = L.sb.vlen;
  L.s_inv.alloc(tile_elems(L.sb));
  tiles_init_padding(L.sb, L.s_inv.p, s);
  galerkin_tiles(c, X, L.sb, L.s_inv.p, s);
  unit_empty_gradient_blocks(L.sb, ls, d.nsub, L.s_inv.p, s);
  DevBuf<double> ws;
  ws.alloc(spd_workspace_elems(L.sb));
  spd_invert(L.sb, L.s_inv.p, ws.p, c->d_err.p, s);
  check_device_error(c, s);
  // column-tetrahedron lists kept for the curl-route products G^T A x
  tet_operators(c, L.tcurl, L.tmass, s);
  {
    std::vector<int32_t> csub(X.mat.begin(), X.mat.end());
    std::vector<int64_t> cout(X.mat.size());
    for (size_t a = 0; a < X.mat.size(); ++a) cout[a] = L.sb.voff[X.mat[a]] + X.loc[a];
    L.col_sub.upload(csub, s);
    L.col_out.upload(cout, s);
  }
  auto local_indices = [&](const std::vector<int64_t> &ctp, const std::vector<int32_t> &ctt,
                           DevBuf<int32_t> &out) {
    const Topology &t = c->topo;
    std::vector<int32_t> li(ctt.size() * 6, -1);
    for (size_t a = 0; a + 1 < ctp.size(); ++a) {
      const int m = X.mat[a];
      const int32_t *nb = d.N_idx.data() + d.N_off[m], *ne = d.N_idx.data() + d.N_off[m + 1];
      for (int64_t e = ctp[a]; e < ctp[a + 1]; ++e)
        for (int q = 0; q < 6; ++q) {
          const int32_t dof = t.edge_dof[t.tet_edges[(int64_t)ctt[e] * 6 + q]];
          if (dof < 0) continue;
          const int32_t *it = std::lower_bound(nb, ne, dof);
          if (it != ne && *it == dof) li[e * 6 + q] = (int32_t)(it - nb);
        }
    }
    out.upload(li, s);
  };
  {
    std::vector<int64_t> ctp;
    std::vector<int32_t> ctt;
    coltet_build(c, X, ctp, ctt, L.ctp_d, L.ctt_d, L.ct_d, s);
    local_indices(ctp, ctt, L.lidx_d);
  }
  {
    // rows -> tetrahedra containing them, with local edge and vertex indices
    const Topology &t = c->topo;
    const int64_t n = t.ndofs(), nt = t.ntets();
    std::vector<int64_t> tp(n + 1, 0);
    for (int64_t q = 0; q < nt * 6; ++q) {
      const int32_t dd = t.edge_dof[t.tet_edges[q]];
      if (dd >= 0) tp[dd + 1]++;
    }
    for (int64_t e = 0; e < n; ++e) tp[e + 1] += tp[e];
    std::vector<int32_t> tl(tp[n]);
    std::vector<int8_t> tpos(tp[n]);
    {
      std::vector<int64_t> fill(tp.begin(), tp.end() - 1);
      for (int64_t q = 0; q < nt * 6; ++q) {
        const int32_t dd = t.edge_dof[t.tet_edges[q]];
        if (dd >= 0) {
          tpos[fill[dd]] = (int8_t)(q % 6);
          tl[fill[dd]++] = (int32_t)(q / 6);
        }
      }
    }
    std::vector<int64_t> rp(1, 0);
    std::vector<int32_t> rt, rl, rv;
    std::vector<int8_t> ps;
    for (int m = 0; m < d.nsub; ++m) {
      const int32_t *nb = d.N_idx.data() + d.N_off[m], *ne = d.N_idx.data() + d.N_off[m + 1];
      const int32_t *vb = ls.xv_vert.data() + ls.xv_off[m], *ve = ls.xv_vert.data() + ls.xv_off[m + 1];
      for (int64_t r = 0; r < d.ni(m); ++r) {
        const int32_t dof = nb[r];
        for (int64_t q = tp[dof]; q < tp[dof + 1]; ++q) {
          const int32_t T = tl[q];
          rt.push_back(T);
          ps.push_back(tpos[q]);
          for (int f = 0; f < 6; ++f) {
            const int32_t df = t.edge_dof[t.tet_edges[(int64_t)T * 6 + f]];
            int32_t li = -1;
            if (df >= 0) {
              const int32_t *it = std::lower_bound(nb, ne, df);
              if (it != ne && *it == df) li = (int32_t)(it - nb);
            }
            rl.push_back(li);
          }
          for (int vq = 0; vq < 4; ++vq) {
            const int32_t v = t.tets[(int64_t)T * 4 + vq];
            const int32_t *it = std::lower_bound(vb, ve, v);
            rv.push_back((it != ve && *it == v) ? (int32_t)(it - vb) : -1);
          }
        }
        rp.push_back((int64_t)rt.size());
      }
    }
    L.rptr.upload(rp, s);
    L.rtet.upload(rt, s);
    L.rpos.upload(ps, s);
    L.rlidx.upload(rl, s);
    L.rvidx.upload(rv, s);
  }
  X.neumann = true;
  {
    std::vector<int64_t> ctp;
    std::vector<int32_t> ctt;
    coltet_build(c, X, ctp, ctt, L.ctp_n, L.ctt_n, L.ct_n, s);
    local_indices(ctp, ctt, L.lidx_n);
  }
  L.sn_inv.alloc(tile_elems(L.sb));
  tiles_init_padding(L.sb, L.sn_inv.p, s);
  galerkin_tiles(c, X, L.sb, L.sn_inv.p, s);
  unit_empty_gradient_blocks(L.sb, ls, d.nsub, L.sn_inv.p, s);
  spd_invert(L.sb, L.sn_inv.p, ws.p, c->d_err.p, s);
  check_device_error(c, s);
  L.sb.schedule(c->sm_count, s);
}

void geneo_eigenvectors(geneo_ctx *c) {
  cudaStream_t s = c->stream;
  if (!c->xi) {
    c->xi.reset(new XiOp());
    build_xi_operator(c, *c->xi, s);
  }
  Lobpcg L(c, s, *c->xi);
  L.nsub = c->dec.nsub;
  L.k = c->opt.lobpcg_block;
  const int k = L.k;
  L.ld = std::max(3 * k, 64);
  L.vlen = c->loc.vlen;
  for (auto *b : {&L.X, &L.LX, &L.BX, &L.W, &L.LW, &L.BW, &L.P, &L.LP, &L.BP, &L.R, &L.T1, &L.T2,
                  &L.T3}) {
    b->alloc(L.vlen * k);
    b->zero(s);
  }
  for (auto *b : {&L.U1, &L.U2}) {
    b->alloc(L.op.vlenS * k);
    b->zero(s);
  }
  L.gram.alloc((int64_t)L.nsub * L.ld * L.ld);
  L.tmat.alloc((int64_t)L.nsub * L.ld * L.ld);
  L.coef.alloc((int64_t)L.nsub * L.ld * L.ld);
  L.theta.alloc((int64_t)L.nsub * k);
  L.nq.assign(L.nsub, 0);
  grow_q(L, 16);
  // search-direction operator: A_j^-1, or (A_j^Neu + 1e-10 diag)^-1 for
  // lobpcg_neumann and for the classical pencil (whose top eigenvectors carry
  // large components on the dofs outside the partition of unity's support,
  // where only B = A_j^Neu couples them: with A_j^-1 directions the
  // residuals stall near 1e-2 while the Ritz values settle)
  const bool neu = c->opt.lobpcg_neumann != 0;
  const bool neu_dir = neu || c->opt.geneo_pencil == GENEO_PENCIL_CLASSICAL;
  DevBuf<double> neu_inv;
  if (neu_dir) {
    neu_inv.alloc(tile_elems(c->loc));
    tiles_init_padding(c->loc, neu_inv.p, s);
    k_neumann_tiles<<<dim3(64, L.nsub), 256, 0, s>>>(L.op.Noff.p, L.op.lrp.p, L.op.lcol.p,
                                                      L.op.nval.p, c->loc.d_toff.p, 1e-10,
                                                      neu_inv.p);
    GENEO_CHECK_LAUNCH();
    DevBuf<double> ws;
    ws.alloc(spd_workspace_elems(c->loc));
    spd_invert(c->loc, neu_inv.p, ws.p, c->d_err.p, s);
    check_device_error(c, s);
  }
  const double *Tdir = neu_dir ? neu_inv.p : c->loc_f64.p;
  const double tau = c->tau_p, tol = c->opt.lobpcg_tol;
  std::vector<uint8_t> done(L.nsub, 0);
  std::vector<std::vector<double>> lam_locked(L.nsub);
  c->lobpcg_iters.assign(L.nsub, 0);
  c->lobpcg_iters0.assign(L.nsub, 0);
  const int ld = L.ld;
  for (int round = 0;; ++round) {
    bool any = false;
    for (int m = 0; m < L.nsub; ++m) any |= !done[m];
    if (!any) break;
    // fresh block, B-orthogonal to the locked vectors, B-orthonormal; the
    // first block comes from the warm-start network when one is given
    if (round == 0 && c->opt.warm_start)
      mlp_infer(c->opt.warm_start->m, c, L.X.p, s);
    else
      k_rand_block<<<grid_for(L.vlen, 256), 256, 0, s>>>(L.X.p, k, L.vlen, c->d_l2g.p,
                                                         c->opt.seed, (uint64_t)round);
    project_gradients_B(L, L.X.p, k);
    apply_B(L, L.X.p, L.BX.p, k);
    b_orthogonalize(L, L.X, nullptr, nullptr, 0, true, k);
    apply_B(L, L.X.p, L.BX.p, k);
    cholqr(L, L.X, L.BX, nullptr, k);
    apply_L(L, L.X.p, L.LX.p, k);
    // Rayleigh-Ritz on X alone
    gram(L, L.X.p, k, L.LX.p, k, L.gram.p);
    k_rr_jacobi_cta<<<L.nsub, 256, 0, s>>>(L.gram.p, k, ld, k, L.theta.p, L.coef.p);
    combine(L, cols(L.X, k, L.vlen), L.coef.p, k, L.T1.p);
    std::swap(L.X.p, L.T1.p);
    combine(L, cols(L.LX, k, L.vlen), L.coef.p, k, L.T1.p);
    std::swap(L.LX.p, L.T1.p);
    combine(L, cols(L.BX, k, L.vlen), L.coef.p, k, L.T1.p);
    std::swap(L.BX.p, L.T1.p);
    bool have_p = false;
    std::vector<uint8_t> finished(L.nsub, 0);
    // stall detection: best largest relative residual of the block so far
    // and the iterations since it last dropped by 10%
    std::vector<double> best(L.nsub, 1e300);
    std::vector<int> stall(L.nsub, 0);
    // lobpcg_neumann: the last kHist Ritz values of every subdomain (ring)
    constexpr int kHist = 6;
    std::vector<double> thist(neu ? (size_t)L.nsub * kHist * k : 0);
    std::vector<int> nhist(L.nsub, 0);
    for (int m = 0; m < L.nsub; ++m) finished[m] = done[m];
    for (int it = 0; it < c->opt.lobpcg_maxit; ++it) {
      k_resid<<<grid_for(L.vlen, 256), 256, 0, s>>>(L.LX.p, L.BX.p, L.theta.p, k, L.op.pos_sub.p,
                                                    L.vlen, L.R.p);
      // residual and B X norms, Ritz values
      gram(L, L.R.p, k, L.R.p, k, L.gram.p);
      std::vector<double> gr = L.gram.download(s);
      gram(L, L.BX.p, k, L.BX.p, k, L.gram.p);
      std::vector<double> gb = L.gram.download(s);
      std::vector<double> th = L.theta.download(s);
      if (std::getenv("GENEO_DEBUG")) {
        gram(L, L.LX.p, k, L.LX.p, k, L.gram.p);
        std::vector<double> gl = L.gram.download(s);
        for (int m = 0; m < std::min(L.nsub, 3); ++m) {
          std::fprintf(stderr, "[lobpcg] round %d it %d sub %d fin %d nq %d |", round, it, m,
                       (int)finished[m], L.nq[m]);
          for (int j = 0; j < k; ++j)
            std::fprintf(stderr, " %.4g(r%.1e,b%.1e,l%.1e)", th[m * k + j],
                         std::sqrt(std::max(gr[(size_t)m * ld * ld + j * ld + j], 0.0)),
                         std::sqrt(std::max(gb[(size_t)m * ld * ld + j * ld + j], 0.0)),
                         std::sqrt(std::max(gl[(size_t)m * ld * ld + j * ld + j], 0.0)));
          std::fprintf(stderr, "\n");
        }
      }
      for (int m = 0; m < L.nsub; ++m) {
        c->lobpcg_iters[m] += !finished[m];
        if (round == 0) c->lobpcg_iters0[m] += !finished[m];
      }
      // lock / finish decisions
      std::vector<int32_t> srcc((size_t)L.nsub * k, -1), dstc((size_t)L.nsub * k, -1);
      bool moves = false;
      int need = 0;
      for (int m = 0; m < L.nsub; ++m) {
        if (finished[m]) continue;
        double worst = 0.0;
        for (int j = 0; j < k; ++j) {
          const double rn = std::sqrt(std::max(gr[(size_t)m * ld * ld + j * ld + j], 0.0));
          const double bn = std::sqrt(std::max(gb[(size_t)m * ld * ld + j * ld + j], 0.0));
          const double sc = std::max(std::fabs(th[m * k + j]), tau) * bn;
          if (bn > 0.0) worst = std::max(worst, rn / sc);
        }
        if (worst < 0.9 * best[m]) {
          best[m] = worst;
          stall[m] = 0;
        } else {
          ++stall[m];
        }
        const double tol_m = stall[m] >= 10 ? std::max(tol, 1e-4) : tol;
        if (neu) {
          double *h = thist.data() + ((size_t)m * kHist + nhist[m] % kHist) * k;
          for (int j = 0; j < k; ++j) h[j] = th[m * k + j];
          ++nhist[m];
        }
        // a Ritz value that has stayed within 1e-4 relative over the last
        // kHist iterations, clear of tau (lobpcg_neumann only)
        auto stagnant = [&](int j) {
          if (!neu || nhist[m] < kHist) return false;
          const double t = th[m * k + j];
          if (!(std::fabs(t - tau) > 1e-2 * tau)) return false;
          double dev = 0;
          for (int q = 0; q < kHist; ++q)
            dev = std::max(dev, std::fabs(thist[((size_t)m * kHist + q) * k + j] - t));
          return dev <= 1e-4 * std::max(std::fabs(t), tau);
        };
        int lead = 0;
        for (int j = 0; j < k; ++j) {
          const double rn = std::sqrt(std::max(gr[(size_t)m * ld * ld + j * ld + j], 0.0));
          const double bn = std::sqrt(std::max(gb[(size_t)m * ld * ld + j * ld + j], 0.0));
          const double sc = std::max(std::fabs(th[m * k + j]), tau) * bn;
          if (rn <= tol_m * sc || bn == 0.0 || stagnant(j)) ++lead;
          else break;
        }
        bool fin = false, stop = false;
        int nlock = 0;
        if (lead == k) {
          for (int j = 0; j < k; ++j) nlock += th[m * k + j] > tau;
          fin = true;
          stop = nlock < k;
        } else if (lead >= 1 && th[m * k + lead - 1] <= tau) {
          for (int j = 0; j < lead; ++j) nlock += th[m * k + j] > tau;
          fin = true;
          stop = true;
        } else if (it + 1 == c->opt.lobpcg_maxit) {
          for (int j = 0; j < lead; ++j) nlock += th[m * k + j] > tau;
          fin = true;
          stop = true;
        }
        if (!fin) continue;
        finished[m] = 1;
        if (stop) done[m] = 1;
        for (int j = 0; j < nlock; ++j) {
          srcc[(size_t)m * k + j] = j;
          dstc[(size_t)m * k + j] = L.nq[m] + j;
          lam_locked[m].push_back(th[m * k + j]);
        }
        if (nlock) moves = true;
        L.nq[m] += nlock;
        need = std::max(need, L.nq[m]);
      }
      if (moves) {
        grow_q(L, need);
        DevBuf<int32_t> ds, dd;
        ds.upload(srcc, s);
        dd.upload(dstc, s);
        k_copy_cols<<<grid_for(L.vlen, 256), 256, 0, s>>>(L.X.p, L.Q.p, L.op.pos_sub.p, ds.p, dd.p, k,
                                                          L.vlen);
        k_copy_cols<<<grid_for(L.vlen, 256), 256, 0, s>>>(L.BX.p, L.BQ.p, L.op.pos_sub.p, ds.p, dd.p,
                                                          k, L.vlen);
        GENEO_CUDA(cudaStreamSynchronize(s));
      }
      bool all = true;
      for (int m = 0; m < L.nsub; ++m) all &= finished[m] != 0;
      if (all) break;
      // W = T R (explicit local inverse), B-orthogonal to Q and X, B-orthonormal.
      // For the filtered pencil with the float32 split built, T = C_j in
      // float32: the B-orthogonal projection that follows removes range(G_j),
      // so P_B A_j^-1 R = P_B (G_j S_j^-1 G_j^T + C_j) R = P_B C_j R, and the
      // float32 SYMV streams half the bytes of the float64 one, which is
      // FP64-ALU-bound (a preconditioner of the eigensolve needs no float64)
      const bool f32_dir = !neu_dir && c->loc_f32.p;
      if (f32_dir) {
        // four columns per pass over the float32 factors
        symv_batch_f32_cols(c->loc, c->loc_f32.p, L.R.p, L.W.p, k, c->d_err.p, s);
      } else {
        for (int col = 0; col < k; ++col)
          symv_batch<double>(c->loc, Tdir, L.R.p + (int64_t)col * L.vlen,
                             L.W.p + (int64_t)col * L.vlen, c->d_err.p, s);
      }
      project_gradients_B(L, L.W.p, k);
      apply_B(L, L.W.p, L.BW.p, k);
      b_orthogonalize(L, L.W, &L.X, &L.BX, k, true, k);
      apply_B(L, L.W.p, L.BW.p, k);
      cholqr(L, L.W, L.BW, nullptr, k);
      apply_L(L, L.W.p, L.LW.p, k);
      if (have_p) {
        // P against X and W (B-inner), then B-orthonormal
        apply_B(L, L.P.p, L.BP.p, k);
        b_orthogonalize(L, L.P, &L.X, &L.BX, k, true, k);
        apply_B(L, L.P.p, L.BP.p, k);
        {
          // against W
          gram(L, L.BW.p, k, L.P.p, k, L.gram.p);
          std::vector<double> hg = L.gram.download(s);
          std::vector<double> cf((size_t)L.nsub * ld * ld, 0.0);
          for (int m = 0; m < L.nsub; ++m)
            for (int j = 0; j < k; ++j) {
              cf[(size_t)m * ld * ld + j * ld + j] = 1.0;
              for (int cc = 0; cc < k; ++cc)
                cf[(size_t)m * ld * ld + (k + j) * ld + cc] = -hg[(size_t)m * ld * ld + j * ld + cc];
            }
          L.coef.upload(cf, s);
          std::vector<const double *> src = cols(L.P, k, L.vlen);
          auto wc = cols(L.W, k, L.vlen);
          src.insert(src.end(), wc.begin(), wc.end());
          combine(L, src, L.coef.p, k, L.T1.p);
          std::swap(L.P.p, L.T1.p);
        }
        apply_B(L, L.P.p, L.BP.p, k);
        cholqr(L, L.P, L.BP, nullptr, k);
        apply_L(L, L.P.p, L.LP.p, k);
      }
      const int ns = have_p ? 3 * k : 2 * k;
      // Rayleigh-Ritz: H = S^T L S with S = [X W P] (B-orthonormal)
      {
        std::vector<double> H((size_t)L.nsub * ld * ld, 0.0);
        const DevBuf<double> *Sb[3] = {&L.X, &L.W, &L.P};
        const DevBuf<double> *LSb[3] = {&L.LX, &L.LW, &L.LP};
        for (int a = 0; a < ns / k; ++a)
          for (int b = 0; b < ns / k; ++b) {
            gram(L, Sb[a]->p, k, LSb[b]->p, k, L.gram.p);
            std::vector<double> g = L.gram.download(s);
            for (int m = 0; m < L.nsub; ++m)
              for (int i = 0; i < k; ++i)
                for (int j = 0; j < k; ++j)
                  H[(size_t)m * ld * ld + (a * k + i) * ld + (b * k + j)] =
                      g[(size_t)m * ld * ld + i * ld + j];
          }
        if (neu) {
          // B-Gram of the basis and the Rayleigh-Ritz step in its
          // B-orthonormalised span (the blocks are B-orthonormalised one
          // against the other by single passes, which the B^-1-like
          // directions of this mode leave far from B-orthonormal)
          std::vector<double> Mg((size_t)L.nsub * ld * ld, 0.0);
          const DevBuf<double> *BSb[3] = {&L.BX, &L.BW, &L.BP};
          for (int a = 0; a < ns / k; ++a)
            for (int b = 0; b < ns / k; ++b) {
              gram(L, Sb[a]->p, k, BSb[b]->p, k, L.gram.p);
              std::vector<double> g = L.gram.download(s);
              for (int m = 0; m < L.nsub; ++m)
                for (int i = 0; i < k; ++i)
                  for (int j = 0; j < k; ++j)
                    Mg[(size_t)m * ld * ld + (a * k + i) * ld + (b * k + j)] =
                        g[(size_t)m * ld * ld + i * ld + j];
            }
          std::vector<double> thh((size_t)L.nsub * k), Cm((size_t)L.nsub * ld * ld);
          general_rr_batch(L.nsub, ns, ld, k, H.data(), Mg.data(), thh.data(), Cm.data());
          L.theta.upload(thh, s);
          L.tmat.upload(Cm, s);
        } else {
          L.coef.upload(H, s);
          k_rr_jacobi_cta<<<L.nsub, 256, 0, s>>>(L.coef.p, ns, ld, k, L.theta.p, L.tmat.p);
        }
      }
      // new X, P and their images
      {
        std::vector<const double *> sx = cols(L.X, k, L.vlen), sw = cols(L.W, k, L.vlen),
                                    sp = cols(L.P, k, L.vlen);
        std::vector<const double *> lx = cols(L.LX, k, L.vlen), lw = cols(L.LW, k, L.vlen),
                                    lp = cols(L.LP, k, L.vlen);
        std::vector<const double *> bx = cols(L.BX, k, L.vlen), bw = cols(L.BW, k, L.vlen),
                                    bp = cols(L.BP, k, L.vlen);
        auto cat = [&](std::vector<const double *> a, const std::vector<const double *> &b,
                       const std::vector<const double *> &c2) {
          a.insert(a.end(), b.begin(), b.end());
          if (have_p) a.insert(a.end(), c2.begin(), c2.end());
          return a;
        };
        // P_new = [W P] C[k:, :]  (zero X rows): build a copy of the
        // coefficients with the X rows cleared
        std::vector<double> tm = L.tmat.download(s);
        std::vector<double> tp = tm;
        for (int m = 0; m < L.nsub; ++m)
          for (int i = 0; i < k; ++i)
            for (int j = 0; j < ld; ++j) tp[(size_t)m * ld * ld + i * ld + j] = 0.0;
        DevBuf<double> cpn;
        cpn.upload(tp, s);
        combine(L, cat(sx, sw, sp), cpn.p, k, L.T1.p);   // P_new
        combine(L, cat(lx, lw, lp), cpn.p, k, L.T2.p);   // LP_new
        combine(L, cat(bx, bw, bp), cpn.p, k, L.T3.p);   // BP_new
        combine(L, cat(sx, sw, sp), L.tmat.p, k, L.R.p);  // X_new (R is free now)
        std::swap(L.P.p, L.T1.p);
        std::swap(L.LP.p, L.T2.p);
        std::swap(L.BP.p, L.T3.p);
        combine(L, cat(lx, lw, lp), L.tmat.p, k, L.T1.p);  // LX_new
        std::swap(L.X.p, L.R.p);
        // L X and B X recomputed from X: the combined images carry the
        // rounding of ||L|| ||W|| (large for high-contrast mu^-1), which
        // stalls the residual far above the tolerance
        apply_L(L, L.X.p, L.LX.p, k);
        apply_B(L, L.X.p, L.BX.p, k);
        have_p = true;
      }
      check_device_error(c, s);
    }
  }
  // GenEO columns: R_j^T D_j (I - xi_j) Q_jq, per subdomain in descending
  // lambda order
  int maxq = 0;
  for (int v : L.nq) maxq = std::max(maxq, v);
  c->geneo_found.assign(L.nsub, 0);
  for (int m = 0; m < L.nsub; ++m) c->geneo_found[m] = L.nq[m];
  if (c->opt.keep_eigvecs) {
    // training targets of the warm-start network: the first 8 locked
    // eigenvectors of every subdomain (B-orthonormal) and B times them
    const int qc = std::min(maxq, 8);
    c->eigV.alloc(8 * L.vlen);
    c->eigBV.alloc(8 * L.vlen);
    c->eigV.zero(s);
    c->eigBV.zero(s);
    if (qc > 0) {
      GENEO_CUDA(cudaMemcpyAsync(c->eigV.p, L.Q.p, sizeof(double) * L.vlen * qc,
                                 cudaMemcpyDeviceToDevice, s));
      GENEO_CUDA(cudaMemcpyAsync(c->eigBV.p, L.BQ.p, sizeof(double) * L.vlen * qc,
                                 cudaMemcpyDeviceToDevice, s));
    }
    c->eig_nq.assign(L.nsub, 0);
    for (int m = 0; m < L.nsub; ++m) c->eig_nq[m] = std::min(L.nq[m], 8);
    GENEO_CUDA(cudaStreamSynchronize(s));
  }
  if (maxq == 0) return;
  DevBuf<double> V;
  V.alloc(L.vlen * maxq);
  // process in chunks of k columns through the xi operator
  std::vector<double> hv((size_t)L.vlen * maxq);
  for (int c0 = 0; c0 < maxq; c0 += k) {
    const int kk = std::min(k, maxq - c0);
    GENEO_CUDA(cudaMemsetAsync(L.T2.p, 0, sizeof(double) * L.vlen * k, s));
    GENEO_CUDA(cudaMemcpyAsync(L.T2.p, L.Q.p + (int64_t)c0 * L.vlen, sizeof(double) * L.vlen * kk,
                               cudaMemcpyDeviceToDevice, s));
    if (classical_pencil(L))  // R_j^T D_j V
      GENEO_CUDA(cudaMemcpyAsync(L.T1.p, L.T2.p, sizeof(double) * L.vlen * k,
                                 cudaMemcpyDeviceToDevice, s));
    else  // R_j^T D_j (I - xi_j) V
      xi_apply(L, L.T2.p, L.T1.p, k, 1);
    k_dscale<<<grid_for(L.vlen, 256), 256, 0, s>>>(L.op.dmask.p, kk, L.vlen, L.T1.p,
                                                   V.p + (int64_t)c0 * L.vlen);
  }
  GENEO_CUDA(cudaMemcpyAsync(hv.data(), V.p, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost, s));
  GENEO_CUDA(cudaStreamSynchronize(s));
  const Decomposition &d = c->dec;
  for (int m = 0; m < L.nsub; ++m) {
    std::vector<int> order(L.nq[m]);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return lam_locked[m][a] > lam_locked[m][b]; });
    for (int q : order) {
      c->geneo_sub.push_back(m);
      c->geneo_lambda.push_back(lam_locked[m][q]);
      for (int64_t r = 0; r < d.ni(m); ++r) {
        const int32_t dof = d.N_idx[d.N_off[m] + r];
        if (d.owner[dof] != m) continue;
        c->zc_row.push_back(dof);
        c->zc_val.push_back(hv[(size_t)q * L.vlen + c->loc.voff[m] + r]);
      }
      c->zc_ptr.push_back((int64_t)c->zc_row.size());
    }
  }
  c->n0_geneo = (int64_t)c->geneo_sub.size();
  c->n0 = c->n0_snk + c->n0_geneo;
}

void build_split_factors(geneo_ctx *c) {
  cudaStream_t s = c->stream;
  if (!c->xi) {
    c->xi.reset(new XiOp());
    build_xi_operator(c, *c->xi, s);
  }
  XiOp &op = *c->xi;
  c->loc_f32.alloc(tile_elems(c->loc));
  const int64_t maxT = (int64_t)c->loc.maxnt * (c->loc.maxnt + 1) / 2;
  k_split_cast<<<dim3((unsigned)maxT, c->loc.nmat), 256, 0, s>>>(
      c->loc_f64.p, c->loc.d_nt.p, c->loc.d_toff.p, op.Noff.p, op.ghead.p, op.gtail.p,
      op.s_inv.p, op.sb.d_toff.p, op.shifted ? op.gfac.p : nullptr, c->loc_f32.p);
  GENEO_CHECK_LAUNCH();
  op.u1.alloc(op.vlenS);
  op.u2.alloc(op.vlenS);
  op.u1.zero(s);
  op.u2.zero(s);
  // S_j^-1 in float32 as well, for geneo_use_gradient_precision
  op.s_inv32.alloc(tile_elems(op.sb));
  tiles_cast_f32(op.sb, op.s_inv.p, op.s_inv32.p, s);
  GENEO_CUDA(cudaStreamSynchronize(s));
}

// yl += G_j S_j^-1 G_j^T xl for every subdomain (float64 gradient part of the
// split local inverse), on padded local vectors
void apply_neumann(geneo_ctx *c, const double *x, double *y, int k, cudaStream_t s) {
  XiOp &op = *c->xi;
  k_local_csr<<<grid_for(op.nslots * k, 256), 256, 0, s>>>(op.lrp.p, op.lcol.p, op.nval.p,
                                                           op.slot_sub.p, op.Noff.p,
                                                           c->loc.d_voff.p, op.nslots, k,
                                                           c->loc.vlen, x, y);
  GENEO_CHECK_LAUNCH();
}

void split_gradient_apply(geneo_ctx *c, const double *xl, double *yl, cudaStream_t s, int k,
                          const double *scale) {
  XiOp &op = *c->xi;
  k_gt<<<grid_for(op.nv * k, 256), 256, 0, s>>>(op.sptr.p, op.srow.p, op.ssgn.p, op.vslot_sub.p,
                                                op.xvoff.p, c->loc.d_voff.p, op.sb.d_voff.p, op.nv,
                                                k, op.vlen, op.vlenS, xl, op.u1.p);
  // S_j^-1 in float32 when selected (not with the shift's scale): S_j^-1 is
  // SPD and its rounding stays inside range(G_j), so the split inverse stays
  // SPD (x^T C_j x > 0 on ker G_j^T, and the gradient part is PSD)
  const bool f32 = c->grad32 && op.s_inv32.p && !scale;
  for (int j = 0; j < k; ++j) {
    if (f32)
      symv_batch<float>(op.sb, op.s_inv32.p, op.u1.p + j * op.vlenS, op.u2.p + j * op.vlenS,
                        c->d_err.p, s);
    else
      symv_batch<double>(op.sb, op.s_inv.p, op.u1.p + j * op.vlenS, op.u2.p + j * op.vlenS,
                         c->d_err.p, s);
  }
  k_g<<<grid_for(op.nslots * k, 256), 256, 0, s>>>(op.ghead.p, op.gtail.p, op.slot_sub.p,
                                                   op.Noff.p, c->loc.d_voff.p, op.sb.d_voff.p,
                                                   op.nslots, k, op.vlen, op.vlenS, op.u2.p,
                                                   nullptr, yl, 2, scale);
  GENEO_CHECK_LAUNCH();
}

// bfloat16 split local solve on the tensor cores in the two-sided form
// C_j = (I - xi_j) A_j^-1 (I - xi_j)^T (equal to (I - xi_j) A_j^-1, since
// (I - xi_j) A_j^-1 = A_j^-1 (I - xi_j)^T and the projection is idempotent):
//   u = S_j^-1 G_j^T x,   x' = x - A_j G_j u = (I - xi_j)^T x,
//   v = C_j x' (bfloat16, tensor cores),
//   y = v - G_j S_j^-1 G_j^T A_j v + G_j u.
// The bfloat16 C_j never sees the gradient-type part of the residual, and
// its rounding error is removed from the gradient directions of the output,
// so the perturbation stays in the complement where A_j is not small.
void split_tc_apply(geneo_ctx *c, const double *xl, double *yl, double *xp, cudaStream_t s, int k,
                    cudaEvent_t e0, cudaEvent_t e1) {
  XiOp &op = *c->xi;
  k_gt<<<grid_for(op.nv * k, 256), 256, 0, s>>>(op.sptr.p, op.srow.p, op.ssgn.p, op.vslot_sub.p,
                                                op.xvoff.p, c->loc.d_voff.p, op.sb.d_voff.p, op.nv,
                                                k, op.vlen, op.vlenS, xl, op.u1.p);
  for (int j = 0; j < k; ++j)
    symv_batch<double>(op.sb, op.s_inv.p, op.u1.p + j * op.vlenS, op.u2.p + j * op.vlenS,
                       c->d_err.p, s);
  k_agw<<<grid_for(op.nslots * k, 256), 256, 0, s>>>(
      op.rptr.p, op.rtet.p, op.rpos.p, op.rlidx.p, op.rvidx.p, op.tcurl.p, op.tmass.p,
      op.slot_sub.p, op.Noff.p, c->loc.d_voff.p, op.sb.d_voff.p, op.nslots, k, op.vlen, op.vlenS,
      op.u2.p, xl, xp);
  tc_symm(c, xp, yl, k, s, e0, e1);
  k_gtA_curl<<<grid_for(op.nv * k, 128), 128, 0, s>>>(
      op.ctp_d.p, op.ctt_d.p, op.ct_d.p, op.lidx_d.p, op.tcurl.p, op.tmass.p, op.col_sub.p,
      op.col_out.p, c->loc.d_voff.p, op.nv, k, op.vlen, op.vlenS, yl, op.u1.p);
  for (int j = 0; j < k; ++j)
    symv_batch<double>(op.sb, op.s_inv.p, op.u1.p + j * op.vlenS, op.u3.p + j * op.vlenS,
                       c->d_err.p, s);
  k_sub<<<grid_for(op.vlenS * k, 256), 256, 0, s>>>(op.u2.p, op.u3.p, op.u3.p, op.vlenS * k);
  k_g<<<grid_for(op.nslots * k, 256), 256, 0, s>>>(op.ghead.p, op.gtail.p, op.slot_sub.p,
                                                   op.Noff.p, c->loc.d_voff.p, op.sb.d_voff.p,
                                                   op.nslots, k, op.vlen, op.vlenS, op.u3.p,
                                                   nullptr, yl, 2, nullptr);
  GENEO_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// Gradient shift of the local matrices.  For tiny gamma the gradients of
// Omega_j make A_j numerically singular (kappa ~ 1/(gamma u) and beyond), so
// no float64 factorisation of A_j is meaningful.  With xi_j = G S^-1 G^T A_j
// (Sec. 2, lemma with eq. "inverseBw") and any rho > 0,
//   A~_j = A_j + rho A_j G S^-1 G^T A_j = A_j (I + rho xi_j),
//   A~_j^-1 = (I + rho xi_j)^-1 A_j^-1 = A_j^-1 - rho/(1+rho) G S^-1 G^T,
// since xi_j is a projection.  A~_j lifts only the gradient modes (by 1 + rho),
// so it is factored instead, and exactly
//   C_j = (I - xi_j) A_j^-1 = A~_j^-1 - 1/(1+rho) G S^-1 G^T,
//   A_j^-1 = A~_j^-1 + rho/(1+rho) G S^-1 G^T.
// rho_j puts the mean Rayleigh quotient of the lifted gradient columns at the
// mean diagonal of A_j: rho = (tr A_j / n_j) / (tr H_j / nv_j), H = A G S^-1 G^T A.

namespace {

// w[c][voffS[m] + c] = 1 for the nv_m kept vertices of subdomain m
__global__ void k_ident_cols(const int64_t *__restrict__ xvoff, const int64_t *__restrict__ voffS,
                             int64_t vlenS, double *__restrict__ w) {
  const int m = blockIdx.x;
  const int64_t nv = xvoff[m + 1] - xvoff[m];
  for (int64_t c = threadIdx.x; c < nv; c += blockDim.x) w[c * vlenS + voffS[m] + c] = 1.0;
}

// T[v][rows of tile I] = sum_u AG[u][rows] S^-1(u, v), 64 x 64 output tile
// (I, V) of subdomain m per CTA; columns of length vlen per vertex
__global__ void __launch_bounds__(256) k_ag_sinv(const double *__restrict__ AG,
                                                 const double *__restrict__ sinv,
                                                 const int32_t *__restrict__ nt,
                                                 const int64_t *__restrict__ voff,
                                                 const int32_t *__restrict__ ntS,
                                                 const int64_t *__restrict__ toffS, int64_t vlen,
                                                 double *__restrict__ T) {
  __shared__ double As[kTile * kLd], Bs[kTile * kLd];
  const int m = blockIdx.z, I = blockIdx.x, V = blockIdx.y;
  if (I >= nt[m] || V >= ntS[m]) return;
  const int64_t rb = voff[m] + (int64_t)I * kTile;
  double acc[4][4] = {};
  for (int U = 0; U < ntS[m]; ++U) {
    for (int e = threadIdx.x; e < kTileElems; e += blockDim.x) {
      const int uu = e >> 6, r = e & 63;  // coalesced over rows
      As[r * kLd + uu] = AG[((int64_t)U * kTile + uu) * vlen + rb + r];
      const int a = e >> 6, b = e & 63;   // S^-1(U*64 + a, V*64 + b) -> Bs[b][a]
      double v;
      if (U >= V)
        v = sinv[(toffS[m] + (int64_t)U * (U + 1) / 2 + V) * kTileElems + a * kTile + b];
      else
        v = sinv[(toffS[m] + (int64_t)V * (V + 1) / 2 + U) * kTileElems + b * kTile + a];
      Bs[b * kLd + a] = v;
    }
    __syncthreads();
    gemm_abt(As, Bs, acc);
    __syncthreads();
  }
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      T[((int64_t)V * kTile + tc + 16 * j) * vlen + rb + 4 * tr + i] = acc[i][j];
}

// per subdomain (one CTA): tr A_m over its n_m rows and tr H_m = sum_v T[v] . AG[v]
__global__ void k_shift_rho(const double *__restrict__ ainv, const int64_t *__restrict__ toff,
                            const int64_t *__restrict__ Noff, const int64_t *__restrict__ voff,
                            const int64_t *__restrict__ xvoff, const double *__restrict__ AG,
                            const double *__restrict__ T, int64_t vlen, double *__restrict__ rho,
                            double *__restrict__ gfac, double *__restrict__ gsc) {
  __shared__ double sa[256], sh[256];
  const int m = blockIdx.x;
  const int64_t n = Noff[m + 1] - Noff[m], nv = xvoff[m + 1] - xvoff[m];
  double ta = 0, th = 0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const int64_t I = r / kTile;
    ta += ainv[(toff[m] + I * (I + 1) / 2 + I) * kTileElems + (r % kTile) * (kTile + 1)];
    for (int64_t v = 0; v < nv; ++v) th = fma(T[v * vlen + voff[m] + r], AG[v * vlen + voff[m] + r], th);
  }
  sa[threadIdx.x] = ta;
  sh[threadIdx.x] = th;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sa[threadIdx.x] += sa[threadIdx.x + o];
      sh[threadIdx.x] += sh[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double r = (nv > 0 && sh[0] > 0) ? (sa[0] / (double)n) / (sh[0] / (double)nv) : 0.0;
    rho[m] = r;
    gfac[m] = 1.0 / (1.0 + r);
    gsc[m] = r / (1.0 + r);
  }
}

// A~(I, J) += rho_m sum_v T[v][rows I] AG[v][rows J], J <= I
__global__ void __launch_bounds__(256) k_shift_update(const double *__restrict__ T,
                                                      const double *__restrict__ AG,
                                                      const int32_t *__restrict__ nt,
                                                      const int64_t *__restrict__ toff,
                                                      const int64_t *__restrict__ voff,
                                                      const int32_t *__restrict__ ntS,
                                                      const double *__restrict__ rho,
                                                      int64_t vlen, double *__restrict__ A) {
  __shared__ double As[kTile * kLd], Bs[kTile * kLd];
  const int m = blockIdx.y;
  const int64_t ntm = nt[m];
  const int64_t q = blockIdx.x;
  if (q >= ntm * (ntm + 1) / 2) return;
  int I, J;
  tile_I_J(q, I, J);
  const int64_t ri = voff[m] + (int64_t)I * kTile, rj = voff[m] + (int64_t)J * kTile;
  double acc[4][4] = {};
  for (int V = 0; V < ntS[m]; ++V) {
    for (int e = threadIdx.x; e < kTileElems; e += blockDim.x) {
      const int vv = e >> 6, r = e & 63;
      const int64_t col = ((int64_t)V * kTile + vv) * vlen;
      As[r * kLd + vv] = T[col + ri + r];
      Bs[r * kLd + vv] = AG[col + rj + r];
    }
    __syncthreads();
    gemm_abt(As, Bs, acc);
    __syncthreads();
  }
  const double rh = rho[m];
  double *dst = A + (toff[m] + q) * kTileElems;
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) dst[(4 * tr + i) * kTile + tc + 16 * j] += rh * acc[i][j];
}

}  // namespace

void apply_gradient_shift(geneo_ctx *c) {
  cudaStream_t s = c->stream;
  if (!c->xi) {
    c->xi.reset(new XiOp());
    build_xi_operator(c, *c->xi, s);
  }
  XiOp &op = *c->xi;
  const int nsub = c->dec.nsub;
  const std::vector<int64_t> &xv = c->ls.xv_off;
  int64_t nvmax = 0;
  for (int m = 0; m < nsub; ++m) nvmax = std::max(nvmax, xv[m + 1] - xv[m]);
  op.rho.alloc(nsub);
  op.gfac.alloc(nsub);
  op.gsc64.alloc(nsub);
  op.shifted = true;
  if (nvmax == 0) {
    op.rho.zero(s);
    std::vector<double> one(nsub, 1.0);
    op.gfac.upload(one, s);
    op.gsc64.zero(s);
    return;
  }
  const int64_t kv = (nvmax + kTile - 1) / kTile * kTile;  // vertex columns, tile padded
  const int64_t vlen = c->loc.vlen, vlenS = op.vlenS;
  DevBuf<double> W, AG, T;
  W.alloc(kv * vlenS);
  W.zero(s);
  k_ident_cols<<<nsub, 128, 0, s>>>(op.xvoff.p, op.sb.d_voff.p, vlenS, W.p);
  // -A_j G e_v for every kept vertex v (curl route; y = 0 in out = y - A G w)
  AG.alloc(kv * vlen);
  AG.zero(s);
  k_agw<<<grid_for(op.nslots * kv, 256), 256, 0, s>>>(
      op.rptr.p, op.rtet.p, op.rpos.p, op.rlidx.p, op.rvidx.p, op.tcurl.p, op.tmass.p,
      op.slot_sub.p, op.Noff.p, c->loc.d_voff.p, op.sb.d_voff.p, op.nslots, (int)kv, vlen, vlenS,
      W.p, AG.p, AG.p);
  GENEO_CHECK_LAUNCH();
  W.release();
  T.alloc(kv * vlen);
  T.zero(s);
  const int maxntS = op.sb.maxnt;
  k_ag_sinv<<<dim3(c->loc.maxnt, maxntS, nsub), 256, 0, s>>>(AG.p, op.s_inv.p, c->loc.d_nt.p,
                                                             c->loc.d_voff.p, op.sb.d_nt.p,
                                                             op.sb.d_toff.p, vlen, T.p);
  GENEO_CHECK_LAUNCH();
  k_shift_rho<<<nsub, 256, 0, s>>>(c->loc_f64.p, c->loc.d_toff.p, op.Noff.p, c->loc.d_voff.p,
                                   op.xvoff.p, AG.p, T.p, vlen, op.rho.p, op.gfac.p, op.gsc64.p);
  GENEO_CHECK_LAUNCH();
  const int64_t maxT = (int64_t)c->loc.maxnt * (c->loc.maxnt + 1) / 2;
  k_shift_update<<<dim3((unsigned)maxT, nsub), 256, 0, s>>>(T.p, AG.p, c->loc.d_nt.p,
                                                           c->loc.d_toff.p, c->loc.d_voff.p,
                                                           op.sb.d_nt.p, op.rho.p, vlen,
                                                           c->loc_f64.p);
  GENEO_CHECK_LAUNCH();
  GENEO_CUDA(cudaStreamSynchronize(s));
}

}  // namespace geneo
