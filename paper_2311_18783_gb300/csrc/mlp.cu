// Learned warm start of the batched local eigensolves (the generalised
// eigenproblems of Sec. 3.2, GEVP "tauthresholdAS"): a 5 -> 128 -> 128 -> 8
// ReLU network maps features of every local edge to the 8 columns of the
// first LOBPCG block.  Weights are used in bfloat16 (a float32 master copy is
// trained with Adam), all arithmetic accumulates in float32.
//
// Features of local edge e of subdomain j (float32, 5 per padded local row):
//   f0 = mean of log10(mu^-1) over the tetrahedra of Omega_j containing e, / 6
//   f1 = min(d(tail), d(head), 8) / 8 with d the hop distance along the edges
//        of Omega_j's tetrahedra to its artificial boundary (vertices shared
//        with an active cell outside Omega_j); 8 without such a boundary
//   f2..f4 = |x_head - x_tail| / ||x_head - x_tail||
// Training loss of subdomain j, X its block (n_j x 8), V its locked
// eigenvectors (B-orthonormal, q_j <= 8), B = A_j^Neu, G = X^T B X:
//   L_j = ||(I - V V^T B) X||^2 / ||X||^2 + 0.1 sum_{a != b} G_ab^2 / (G_aa G_bb)
// (subspace term and B-cosines between the columns, both invariant to the
// scale of B), averaged over the subdomains with q_j > 0.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <random>

#include "setup.hpp"
#include "xi.hpp"

namespace geneo {

namespace {

constexpr int kH = 128, kOut = 8, kIn = 5;
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH,
              oW3 = ob2 + kH, ob3 = oW3 + kOut * kH, kNParam = ob3 + kOut;
constexpr int kEdges = 128;    // edges (threads) per CTA
constexpr int kLdH = kH + 1;   // padded rows of the per-edge activation tiles

__device__ __forceinline__ float wgt(const uint16_t *wb, int i) {
  return __uint_as_float(((uint32_t)wb[i]) << 16);
}

// all parameters (bfloat16 -> float32) into shared memory, in the parameter
// layout W1 b1 W2 b2 W3 b3
__device__ void stage_weights(const uint16_t *__restrict__ wb, float *ws) {
  for (int i = threadIdx.x; i < kNParam; i += blockDim.x) ws[i] = wgt(wb, i);
  __syncthreads();
}

// X[c][p] = network(feat[p]) on valid local rows, 0 on padding
__global__ void __launch_bounds__(kEdges) k_mlp_fwd(const float *__restrict__ feat,
                                                    const int32_t *__restrict__ l2g,
                                                    const uint16_t *__restrict__ wb, int64_t vlen,
                                                    double *__restrict__ X) {
  extern __shared__ float sm[];
  float *ws = sm;                  // kNParam
  float *h1s = sm + kNParam + 8;   // [kEdges][kLdH]
  stage_weights(wb, ws);
  const int t = threadIdx.x;
  const int64_t p = blockIdx.x * (int64_t)kEdges + t;
  const bool ok = p < vlen;
  float f[kIn];
#pragma unroll
  for (int i = 0; i < kIn; ++i) f[i] = ok ? feat[p * kIn + i] : 0.f;
  for (int u = 0; u < kH; ++u) {
    float z = ws[ob1 + u];
#pragma unroll
    for (int i = 0; i < kIn; ++i) z = fmaf(ws[oW1 + u * kIn + i], f[i], z);
    h1s[t * kLdH + u] = fmaxf(z, 0.f);
  }
  float out[kOut];
#pragma unroll
  for (int c = 0; c < kOut; ++c) out[c] = ws[ob3 + c];
  for (int u0 = 0; u0 < kH; u0 += 16) {
    float acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = ws[ob2 + u0 + j];
    for (int k = 0; k < kH; ++k) {
      const float hk = h1s[t * kLdH + k];
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = fmaf(ws[oW2 + (u0 + j) * kH + k], hk, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float h2 = fmaxf(acc[j], 0.f);
#pragma unroll
      for (int c = 0; c < kOut; ++c) out[c] = fmaf(ws[oW3 + c * kH + u0 + j], h2, out[c]);
    }
  }
  if (!ok) return;
  const bool valid = l2g[p] >= 0;
#pragma unroll
  for (int c = 0; c < kOut; ++c) X[(int64_t)c * vlen + p] = valid ? (double)out[c] : 0.0;
}

// partial parameter gradient of sum_p <dX[:, p], network(feat[p])> over the
// CTA's 128 rows (deterministic loops, one partial vector per CTA)
__global__ void __launch_bounds__(kEdges) k_mlp_bwd(const float *__restrict__ feat,
                                                    const int32_t *__restrict__ l2g,
                                                    const uint16_t *__restrict__ wb, int64_t vlen,
                                                    const double *__restrict__ dX,
                                                    float *__restrict__ part) {
  extern __shared__ float sm[];
  float *ws = sm;                        // kNParam
  float *B = sm + kNParam + 8;           // [e][k]: h1, later dz1
  float *C = B + kEdges * kLdH;          // [e][u]: z2, later dz2
  float *Fs = C + kEdges * kLdH;         // [e][5]
  float *Ds = Fs + kEdges * kIn;         // [e][8]
  stage_weights(wb, ws);
  const int t = threadIdx.x;
  const int64_t p = blockIdx.x * (int64_t)kEdges + t;
  const bool ok = p < vlen && l2g[p] >= 0;
  for (int i = 0; i < kIn; ++i) Fs[t * kIn + i] = ok ? feat[p * kIn + i] : 0.f;
  for (int c = 0; c < kOut; ++c) Ds[t * kOut + c] = ok ? (float)dX[(int64_t)c * vlen + p] : 0.f;
  // forward: h1 -> B, z2 -> C
  for (int u = 0; u < kH; ++u) {
    float z = ws[ob1 + u];
    for (int i = 0; i < kIn; ++i) z = fmaf(ws[oW1 + u * kIn + i], Fs[t * kIn + i], z);
    B[t * kLdH + u] = fmaxf(z, 0.f);
  }
  for (int u0 = 0; u0 < kH; u0 += 16) {
    float acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = ws[ob2 + u0 + j];
    for (int k = 0; k < kH; ++k) {
      const float hk = B[t * kLdH + k];
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = fmaf(ws[oW2 + (u0 + j) * kH + k], hk, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) C[t * kLdH + u0 + j] = acc[j];
  }
  __syncthreads();
  float *pc = part + (int64_t)blockIdx.x * kNParam;
  // dW3[c][u] = sum_e D[e][c] relu(z2[e][u]) (thread = u); db3
  {
    float a[kOut];
    for (int c = 0; c < kOut; ++c) a[c] = 0.f;
    for (int e = 0; e < kEdges; ++e) {
      const float h2 = fmaxf(C[e * kLdH + t], 0.f);
      for (int c = 0; c < kOut; ++c) a[c] = fmaf(Ds[e * kOut + c], h2, a[c]);
    }
    for (int c = 0; c < kOut; ++c) pc[oW3 + c * kH + t] = a[c];
    if (t < kOut) {
      float s = 0.f;
      for (int e = 0; e < kEdges; ++e) s += Ds[e * kOut + t];
      pc[ob3 + t] = s;
    }
  }
  __syncthreads();
  // dz2[e][u] = (sum_c W3[c][u] D[e][c]) [z2 > 0] (thread = e, own row)
  for (int u = 0; u < kH; ++u) {
    float g = 0.f;
    for (int c = 0; c < kOut; ++c) g = fmaf(ws[oW3 + c * kH + u], Ds[t * kOut + c], g);
    C[t * kLdH + u] = C[t * kLdH + u] > 0.f ? g : 0.f;
  }
  __syncthreads();
  // dW2[u][k] = sum_e dz2[e][u] h1[e][k] (thread = u); db2
  for (int k0 = 0; k0 < kH; k0 += 32) {
    float a[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) a[j] = 0.f;
    for (int e = 0; e < kEdges; ++e) {
      const float d = C[e * kLdH + t];
#pragma unroll
      for (int j = 0; j < 32; ++j) a[j] = fmaf(d, B[e * kLdH + k0 + j], a[j]);
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) pc[oW2 + t * kH + k0 + j] = a[j];
  }
  {
    float s = 0.f;
    for (int e = 0; e < kEdges; ++e) s += C[e * kLdH + t];
    pc[ob2 + t] = s;
  }
  __syncthreads();
  // dz1[e][k] = (sum_u W2[u][k] dz2[e][u]) [h1 > 0] (thread = e, own row of B)
  for (int k = 0; k < kH; ++k) {
    float g = 0.f;
    for (int u = 0; u < kH; ++u) g = fmaf(ws[oW2 + u * kH + k], C[t * kLdH + u], g);
    B[t * kLdH + k] = B[t * kLdH + k] > 0.f ? g : 0.f;
  }
  __syncthreads();
  // dW1[u][i] = sum_e dz1[e][u] f[e][i]; db1 (thread = u)
  {
    float a[kIn + 1];
    for (int i = 0; i <= kIn; ++i) a[i] = 0.f;
    for (int e = 0; e < kEdges; ++e) {
      const float d = B[e * kLdH + t];
      for (int i = 0; i < kIn; ++i) a[i] = fmaf(d, Fs[e * kIn + i], a[i]);
      a[kIn] += d;
    }
    for (int i = 0; i < kIn; ++i) pc[oW1 + t * kIn + i] = a[i];
    pc[ob1 + t] = a[kIn];
  }
}

// grad[i] = sum over CTAs of part[cta][i], in CTA order
__global__ void k_sum_parts(const float *__restrict__ part, int nparts, float *__restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParam) return;
  double s = 0;
  for (int q = 0; q < nparts; ++q) s += part[(int64_t)q * kNParam + i];
  grad[i] = (float)s;
}

// Adam step and the bfloat16 copy of the weights
__global__ void k_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, float lr, float b1t, float b2t,
                       uint16_t *__restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParam) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  m[i] = b1 * m[i] + (1.f - b1) * g[i];
  v[i] = b2 * v[i] + (1.f - b2) * g[i] * g[i];
  const float mh = m[i] / (1.f - b1t), vh = v[i] / (1.f - b2t);
  w[i] -= lr * mh / (sqrtf(vh) + eps);
  wb[i] = __bfloat16_as_ushort(__float2bfloat16_rn(w[i]));
}

__global__ void k_to_bf16(const float *__restrict__ w, uint16_t *__restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kNParam) wb[i] = __bfloat16_as_ushort(__float2bfloat16_rn(w[i]));
}

// Subspace loss of subdomain m (one CTA) and dX on its rows; weight w_m =
// 1/J for subdomains with eigenvectors (q_m > 0), 0 otherwise.
// X, BX: [8][vlen]; V, BV: [8][vlen] (columns >= q_m unused)
__global__ void __launch_bounds__(256) k_subspace_loss(
    const double *__restrict__ X, const double *__restrict__ BX, const double *__restrict__ V,
    const double *__restrict__ BV, const int32_t *__restrict__ nq, const int64_t *__restrict__ voff,
    const int64_t *__restrict__ Noff, int64_t vlen, double inv_j, double *__restrict__ loss,
    double *__restrict__ dX) {
  __shared__ double red[256];
  __shared__ double Gxx[kOut * kOut], Gvx[kOut * kOut], Gvx_keep[kOut * kOut], Gvr[kOut * kOut],
      sc[4];
  const int m = blockIdx.x, q = nq[m];
  const int64_t vb = voff[m], n = Noff[m + 1] - Noff[m];
  const int t = threadIdx.x;
  auto block_sum = [&](double v) {
    red[t] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (t < o) red[t] += red[t + o];
      __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
  };
  if (q == 0) {
    for (int64_t r = t; r < n; r += blockDim.x)
      for (int c = 0; c < kOut; ++c) dX[(int64_t)c * vlen + vb + r] = 0.0;
    if (t == 0) loss[m] = 0.0;
    return;
  }
  // X^T B X, V^T B X, ||X||^2
  for (int a = 0; a < kOut; ++a)
    for (int b = 0; b < kOut; ++b) {
      double s = 0;
      for (int64_t r = t; r < n; r += blockDim.x)
        s = fma(X[(int64_t)a * vlen + vb + r], BX[(int64_t)b * vlen + vb + r], s);
      s = block_sum(s);
      if (t == 0) Gxx[a * kOut + b] = s;
    }
  for (int i = 0; i < q; ++i)
    for (int a = 0; a < kOut; ++a) {
      double s = 0;
      for (int64_t r = t; r < n; r += blockDim.x)
        s = fma(V[(int64_t)i * vlen + vb + r], BX[(int64_t)a * vlen + vb + r], s);
      s = block_sum(s);
      if (t == 0) Gvx[i * kOut + a] = s;
    }
  {
    double s = 0;
    for (int64_t r = t; r < n; r += blockDim.x)
      for (int a = 0; a < kOut; ++a) {
        const double x = X[(int64_t)a * vlen + vb + r];
        s = fma(x, x, s);
      }
    s = block_sum(s);
    if (t == 0) sc[0] = s;
  }
  __syncthreads();
  for (int e = t; e < kOut * kOut; e += blockDim.x) Gvx_keep[e] = Gvx[e];
  __syncthreads();
  // R = X - V Gvx (recomputed per row); ||R||^2 and V^T R
  auto Rval = [&](int a, int64_t r) {
    double v = X[(int64_t)a * vlen + vb + r];
    for (int i = 0; i < q; ++i) v -= V[(int64_t)i * vlen + vb + r] * Gvx[i * kOut + a];
    return v;
  };
  {
    double s = 0;
    for (int64_t r = t; r < n; r += blockDim.x)
      for (int a = 0; a < kOut; ++a) {
        const double v = Rval(a, r);
        s = fma(v, v, s);
      }
    s = block_sum(s);
    if (t == 0) sc[1] = s;
  }
  for (int i = 0; i < q; ++i)
    for (int a = 0; a < kOut; ++a) {
      double s = 0;
      for (int64_t r = t; r < n; r += blockDim.x)
        s = fma(V[(int64_t)i * vlen + vb + r], Rval(a, r), s);
      s = block_sum(s);
      if (t == 0) Gvr[i * kOut + a] = s;
    }
  // B-cosine term and H = dL2/dG: off-diagonal 0.2 G_ab / (d_a d_b),
  // diagonal -0.2 sum_{b != a} G_ab^2 / (d_a^2 d_b)
  if (t == 0) {
    double L2 = 0;
    for (int a = 0; a < kOut; ++a) {
      double hd = 0;
      for (int b = 0; b < kOut; ++b) {
        if (a == b) continue;
        const double g = Gxx[a * kOut + b], dd = Gxx[a * kOut + a] * Gxx[b * kOut + b];
        L2 += g * g / dd;
        Gvx[a * kOut + b] = 0.2 * g / dd;  // Gvx is free now: holds H
        hd -= 0.2 * g * g / (dd * Gxx[a * kOut + a]);
      }
      Gvx[a * kOut + a] = hd;
    }
    sc[2] = 0.1 * L2;
  }
  __syncthreads();
  const double nX = sc[0], L1 = sc[1] / nX;
  if (t == 0) loss[m] = (L1 + sc[2]) * inv_j;
  // dX = [2 (R - B V (V^T R)) / nX - 2 L1 X / nX + 2 B X H] / J
  for (int64_t r = t; r < n; r += blockDim.x)
    for (int a = 0; a < kOut; ++a) {
      double g = X[(int64_t)a * vlen + vb + r];
      for (int i = 0; i < q; ++i) g -= V[(int64_t)i * vlen + vb + r] * Gvx_keep[i * kOut + a];
      for (int i = 0; i < q; ++i) g -= BV[(int64_t)i * vlen + vb + r] * Gvr[i * kOut + a];
      g = 2.0 * g / nX - 2.0 * L1 * X[(int64_t)a * vlen + vb + r] / nX;
      double be = 0;
      for (int b = 0; b < kOut; ++b) be = fma(BX[(int64_t)b * vlen + vb + r], Gvx[b * kOut + a], be);
      dX[(int64_t)a * vlen + vb + r] = (g + 2.0 * be) * inv_j;
    }
}

constexpr size_t kFwdSmem = (size_t)(kNParam + 8 + kEdges * kLdH) * sizeof(float);
constexpr size_t kBwdSmem =
    (size_t)(kNParam + 8 + 2 * kEdges * kLdH + kEdges * kIn + kEdges * kOut) * sizeof(float);

}  // namespace

// ---------------------------------------------------------------------------

struct Mlp {
  DevBuf<float> w, m, v, grad, part;
  DevBuf<uint16_t> wb;
  int64_t step = 0;
  int device = 0;
};

int mlp_param_count() { return kNParam; }

Mlp *mlp_create(uint64_t seed) {
  auto M = new Mlp();
  GENEO_CUDA(cudaGetDevice(&M->device));
  // He-normal weights from a seeded std::mt19937_64 stream, zero biases
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  std::vector<float> w(kNParam, 0.f);
  for (int i = 0; i < kH * kIn; ++i) w[oW1 + i] = (float)(nd(rng) * std::sqrt(2.0 / kIn));
  for (int i = 0; i < kH * kH; ++i) w[oW2 + i] = (float)(nd(rng) * std::sqrt(2.0 / kH));
  for (int i = 0; i < kOut * kH; ++i) w[oW3 + i] = (float)(nd(rng) * std::sqrt(2.0 / kH));
  M->w.upload(w);
  M->m.alloc(kNParam);
  M->v.alloc(kNParam);
  M->m.zero();
  M->v.zero();
  M->grad.alloc(kNParam);
  M->wb.alloc(kNParam);
  k_to_bf16<<<grid_for(kNParam, 256), 256>>>(M->w.p, M->wb.p);
  GENEO_CHECK_LAUNCH();
  GENEO_CUDA(cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kFwdSmem));
  GENEO_CUDA(cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kBwdSmem));
  GENEO_CUDA(cudaDeviceSynchronize());
  return M;
}

void mlp_destroy(Mlp *M) { delete M; }

std::vector<float> mlp_get(const Mlp *M) { return M->w.download(); }

void mlp_set(Mlp *M, const std::vector<float> &w) {
  if ((int64_t)w.size() != kNParam) throw Error(GENEO_ERR_INVALID_ARG, "wrong parameter count");
  GENEO_CUDA(cudaMemcpy(M->w.p, w.data(), sizeof(float) * kNParam, cudaMemcpyHostToDevice));
  M->m.zero();
  M->v.zero();
  M->step = 0;
  k_to_bf16<<<grid_for(kNParam, 256), 256>>>(M->w.p, M->wb.p);
  GENEO_CHECK_LAUNCH();
  GENEO_CUDA(cudaDeviceSynchronize());
}

// X [8][vlen] = network(features) (zero on padding)
void mlp_infer(const Mlp *M, geneo_ctx *c, double *X, cudaStream_t s) {
  if (!c->d_feat.p) throw Error(GENEO_ERR_STATE, "the context has no edge features");
  const int64_t vlen = c->loc.vlen;
  k_mlp_fwd<<<grid_for(vlen, kEdges), kEdges, kFwdSmem, s>>>(c->d_feat.p, c->d_l2g.p, M->wb.p,
                                                             vlen, X);
  GENEO_CHECK_LAUNCH();
}

// loss and parameter gradient on the context's stored eigenvectors; grad
// stays in M->grad
double mlp_loss_grad(Mlp *M, geneo_ctx *c, cudaStream_t s) {
  if (!c->d_feat.p || !c->eigV.p)
    throw Error(GENEO_ERR_STATE, "the context keeps no features or eigenvectors");
  const int64_t vlen = c->loc.vlen;
  const int nsub = c->dec.nsub;
  int J = 0;
  for (int m = 0; m < nsub; ++m) J += c->eig_nq[m] > 0;
  if (J == 0) throw Error(GENEO_ERR_STATE, "no subdomain has eigenvectors");
  DevBuf<double> X, BX, dX, loss;
  X.alloc(kOut * vlen);
  BX.alloc(kOut * vlen);
  dX.alloc(kOut * vlen);
  dX.zero(s);
  loss.alloc(nsub);
  mlp_infer(M, c, X.p, s);
  apply_neumann(c, X.p, BX.p, kOut, s);
  DevBuf<int32_t> dnq;
  dnq.upload(c->eig_nq, s);
  k_subspace_loss<<<nsub, 256, 0, s>>>(X.p, BX.p, c->eigV.p, c->eigBV.p, dnq.p, c->loc.d_voff.p,
                                       c->xi->Noff.p, vlen, 1.0 / J, loss.p, dX.p);
  const unsigned nblk = grid_for(vlen, kEdges);
  if (M->part.n < (int64_t)nblk * kNParam) M->part.alloc((int64_t)nblk * kNParam);
  k_mlp_bwd<<<nblk, kEdges, kBwdSmem, s>>>(c->d_feat.p, c->d_l2g.p, M->wb.p, vlen, dX.p,
                                           M->part.p);
  k_sum_parts<<<grid_for(kNParam, 256), 256, 0, s>>>(M->part.p, (int)nblk, M->grad.p);
  GENEO_CHECK_LAUNCH();
  std::vector<double> l = loss.download(s);
  double tot = 0;
  for (double x : l) tot += x;
  return tot;
}

void mlp_adam(Mlp *M, double lr, cudaStream_t s) {
  ++M->step;
  const float b1t = std::pow(0.9f, (float)M->step), b2t = std::pow(0.999f, (float)M->step);
  k_adam<<<grid_for(kNParam, 256), 256, 0, s>>>(M->w.p, M->m.p, M->v.p, M->grad.p, (float)lr, b1t,
                                                b2t, M->wb.p);
  GENEO_CHECK_LAUNCH();
}

std::vector<float> mlp_grad_host(const Mlp *M, cudaStream_t s) { return M->grad.download(s); }

// ---------------------------------------------------------------------------
// edge features (host integer and coefficient work, once per set-up)

void build_mlp_features(geneo_ctx *c) {
  const Topology &t = c->topo;
  const Decomposition &d = c->dec;
  const int nx = t.nx, ny = t.ny, nz = t.nz;
  const int64_t nverts = t.nverts, vlen = c->loc.vlen;
  std::vector<float> F(vlen * kIn, 0.f);
  std::vector<uint8_t> in_sub(t.ncells, 0), active(t.ncells, 0);
  for (int32_t cl : t.cells) active[cl] = 1;
  std::vector<int> dist(nverts, -1);
  std::vector<int32_t> touched, adj_ptr, adj;
  std::vector<double> acc;
  std::vector<int> cnt;
  for (int m = 0; m < d.nsub; ++m) {
    const int32_t *nb = d.N_idx.data() + d.N_off[m];
    const int64_t n = d.ni(m);
    for (int32_t cl : d.sub_cells[m]) in_sub[cl] = 1;
    acc.assign(n, 0.0);
    cnt.assign(n, 0);
    touched.clear();
    // vertices and edges of Omega_m's tetrahedra
    std::vector<std::pair<int32_t, int32_t>> pairs;
    for (int32_t cl : d.sub_cells[m]) {
      const double lm = std::log10(c->mu_inv[cl]);
      const int64_t r0 = (int64_t)t.cell_rank[cl] * 6;
      for (int64_t tt = r0; tt < r0 + 6; ++tt) {
        for (int q = 0; q < 4; ++q) {
          const int32_t v = t.tets[tt * 4 + q];
          if (dist[v] == -1) {
            dist[v] = 8;
            touched.push_back(v);
          }
        }
        for (int q = 0; q < 6; ++q) {
          const int32_t e = t.tet_edges[tt * 6 + q];
          pairs.push_back({t.edges[2 * e], t.edges[2 * e + 1]});
          const int32_t dof = t.edge_dof[e];
          if (dof < 0) continue;
          const int32_t *it = std::lower_bound(nb, nb + n, dof);
          if (it != nb + n && *it == dof) {
            acc[it - nb] += lm;
            ++cnt[it - nb];
          }
        }
      }
    }
    // adjacency (CSR over the touched vertices, by global id via a map)
    std::sort(touched.begin(), touched.end());
    auto vid = [&](int32_t v) {
      return (int32_t)(std::lower_bound(touched.begin(), touched.end(), v) - touched.begin());
    };
    const int nvl = (int)touched.size();
    std::vector<std::vector<int32_t>> nbr(nvl);
    for (auto &pr : pairs) {
      const int32_t a = vid(pr.first), b = vid(pr.second);
      nbr[a].push_back(b);
      nbr[b].push_back(a);
    }
    // sources: vertices shared with an active cell outside Omega_m
    std::vector<int> dl(nvl, 8);
    std::vector<int32_t> frontier;
    for (int a = 0; a < nvl; ++a) {
      const int32_t v = touched[a];
      const int vi = (int)(v % (nx + 1)), vj = (int)((v / (nx + 1)) % (ny + 1)),
                vk = (int)(v / ((int64_t)(nx + 1) * (ny + 1)));
      bool src = false;
      for (int dk = -1; dk <= 0 && !src; ++dk)
        for (int dj = -1; dj <= 0 && !src; ++dj)
          for (int di = -1; di <= 0 && !src; ++di) {
            const int ci = vi + di, cj = vj + dj, ck = vk + dk;
            if (ci < 0 || cj < 0 || ck < 0 || ci >= nx || cj >= ny || ck >= nz) continue;
            const int64_t cl = ci + (int64_t)nx * (cj + (int64_t)ny * ck);
            if (active[cl] && !in_sub[cl]) src = true;
          }
      if (src) {
        dl[a] = 0;
        frontier.push_back(a);
      }
    }
    std::vector<uint8_t> seen(nvl, 0);
    for (int a : frontier) seen[a] = 1;
    for (int dd = 1; dd <= 8 && !frontier.empty(); ++dd) {
      std::vector<int32_t> nxt;
      for (int a : frontier)
        for (int b : nbr[a])
          if (!seen[b]) {
            seen[b] = 1;
            dl[b] = dd;
            nxt.push_back(b);
          }
      frontier.swap(nxt);
    }
    for (int64_t r = 0; r < n; ++r) {
      const int32_t e = t.dof_edge[nb[r]];
      const int32_t a = t.edges[2 * e], b = t.edges[2 * e + 1];
      const int dmin = std::min(std::min(dl[vid(a)], dl[vid(b)]), 8);
      const int dir = t.edge_dir[e];
      double vx = kDir[dir][0] * t.h[0], vy = kDir[dir][1] * t.h[1], vz = kDir[dir][2] * t.h[2];
      const double nrm = std::sqrt(vx * vx + vy * vy + vz * vz);
      float *f = F.data() + (c->loc.voff[m] + r) * kIn;
      f[0] = (float)(acc[r] / std::max(cnt[r], 1) / 6.0);
      f[1] = (float)(dmin / 8.0);
      f[2] = (float)(std::fabs(vx) / nrm);
      f[3] = (float)(std::fabs(vy) / nrm);
      f[4] = (float)(std::fabs(vz) / nrm);
    }
    for (int32_t v : touched) dist[v] = -1;
    for (int32_t cl : d.sub_cells[m]) in_sub[cl] = 0;
  }
  c->d_feat.upload(F, c->stream);
  GENEO_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace geneo
