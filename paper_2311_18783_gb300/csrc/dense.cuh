// Batched dense symmetric matrices in tile-packed storage, their explicit
// inversion by tiled Cholesky, and the streaming SYMV that applies them.
//
// Storage: matrix m of dimension dim[m] is padded to nt[m] = ceil(dim/64)
// tiles per side; only tiles (I, J) with J <= I are stored, each a full 64x64
// row-major block, at tile index toff[m] + I(I+1)/2 + J.  Diagonal tiles hold
// both triangles.  Padding rows/columns carry an identity diagonal, so the
// factorisation leaves them decoupled.  Vectors use the padded layout: matrix m owns
// elements [voff[m], voff[m] + 64 nt[m]).
#pragma once
#include "common.cuh"

namespace geneo {

// ---- 64x64 tile helpers shared by the dense kernels

// (I, J) of the q-th lower tile in row-major packed order
__device__ __forceinline__ void tile_I_J(int64_t q, int &I, int &J) {
  int i = (int)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
  while ((int64_t)(i + 1) * (i + 2) / 2 <= q) ++i;
  while ((int64_t)i * (i + 1) / 2 > q) --i;
  I = i;
  J = (int)(q - (int64_t)i * (i + 1) / 2);
}

constexpr int kLd = kTile + 1;  // padded shared-memory leading dimension

// acc[i][j] += sum_t As[ri][t] * Bs[cj][t], rows ri = 4*tr + i, cols cj = tc + 16 j
__device__ __forceinline__ void gemm_abt(const double *As, const double *Bs, double acc[4][4]) {
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
#pragma unroll 4
  for (int t = 0; t < kTile; ++t) {
    double a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = As[(4 * tr + i) * kLd + t];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = Bs[(tc + 16 * j) * kLd + t];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
}


// One launch configuration of the streaming SYMV: bulk-copy stages, tiles
// per barrier pair, warps per CTA, persistent CTAs per SM.
struct SymvCfg {
  int nst, d, warps, cps;
};

struct TileBatch {
  int nmat = 0;
  int maxnt = 0;
  std::vector<int32_t> nt;
  std::vector<int64_t> dim, toff, voff;
  int64_t ntiles = 0, vlen = 0;
  DevBuf<int32_t> d_nt;
  DevBuf<int64_t> d_toff, d_voff;
  DevBuf<int32_t> d_vrow_m, d_vrow_I;  // per 64-block of the padded vector
  // SYMV schedule (strips = tile rows, grouped per CTA)
  int sched_ctas = 0;
  DevBuf<int32_t> d_strip_m, d_strip_I, d_cta_off;
  DevBuf<double> rowpart, colpart;   // partial sums of the streaming SYMV
  DevBuf<double> rowpart_nr;         // the same for 4 columns at once (float32 tiles)
  DevBuf<float> colpart_nr;
  // launch configuration per storage type (0 float, 1 double): an index into
  // the candidate lists of the autotuner (0 = default)
  int symv_cfg[2] = {0, 0};
  // schedules with more CTAs per SM (non-owning views plus owned storage)
  struct View {
    int32_t *p = nullptr;
  };
  struct Sched {
    int nctas = 0;
    View strip_m, strip_I, cta_off;
    DevBuf<int32_t> own_m, own_I, own_off;
  };
  int base_ctas = 0;
  Sched base, extra[3];

  void layout(const std::vector<int64_t> &dims);
  void upload_meta(cudaStream_t s);
  void schedule(int nctas, cudaStream_t s);
  const Sched &sched_for(int cps);
};

// -- Explicit inverse of every matrix of the batch, in place (float64), by
// tiled Cholesky, forward substitution on the identity and A^-1 = Y^T Y.
// Pivots that are not positive set err (kDevNotSPD).  ws must hold
// spd_workspace_elems(b) doubles.  Synchronises the stream.
int64_t spd_workspace_elems(const TileBatch &b);
void spd_invert(TileBatch &b, double *data, double *ws, int *d_err, cudaStream_t s);
// Tiled Cholesky of the first nsteps pivot tiles (all when d_npiv is null,
// else npiv[m] per matrix; the trailing tiles then hold the Schur
// complement).  dinv receives L_kk^-1 for every factored diagonal tile at
// tile index dtoff[m] + k.
void chol_factor(TileBatch &b, double *data, const int32_t *d_npiv, int nsteps, double *dinv,
                 const int64_t *d_dtoff, int *d_err, cudaStream_t s);

// Y = L11^-1 for the leading npiv[m] pivot tiles of every matrix (L from
// chol_factor with the same npiv, dinv its inverted diagonal tiles).
void pivot_block_inverse(TileBatch &b, const double *L, double *Y, const double *dinv,
                         const int64_t *d_dtoff, const int32_t *d_npiv, int max_npiv,
                         cudaStream_t s);

// -- y = blockdiag(A_m) x on padded vectors.  Templated on the storage type.
// ev_before / ev_after, when given, are recorded around the streaming kernel.
template <typename T>
void symv_batch(TileBatch &b, const T *data, const double *x, double *y, int *d_err,
                cudaStream_t s, cudaEvent_t ev_before = nullptr, cudaEvent_t ev_after = nullptr);

// y_c = blockdiag(A_m) x_c for nr columns of float32 tiles (x, y: nr padded
// vectors of b.vlen, one after another).  Columns go through the stream four
// at a time, each tile read once per group; column c equals
// symv_batch<float>(x_c) bit for bit under the batch's float configuration.
// ev_before / ev_after, when given, are recorded around the first group's
// streaming kernel (nr >= 4).
void symv_batch_f32_cols(TileBatch &b, const float *data, const double *x, double *y, int nr,
                         int *d_err, cudaStream_t s, cudaEvent_t ev_before = nullptr,
                         cudaEvent_t ev_after = nullptr);

// The autotuner's candidate configurations of symv_batch<T>.
template <typename T> int symv_candidates();
template <typename T> SymvCfg symv_candidate(int idx);

// Pointer/size of a tile-packed buffer in elements.
inline int64_t tile_elems(const TileBatch &b) { return b.ntiles * (int64_t)kTileElems; }

// Fill storage with zeros and an identity diagonal on padding rows.
void tiles_init_padding(TileBatch &b, double *data, cudaStream_t s);
// Cast float64 tile storage to float32.
void tiles_cast_f32(const TileBatch &b, const double *src, float *dst, cudaStream_t s);

int device_sm_count();

}  // namespace geneo
