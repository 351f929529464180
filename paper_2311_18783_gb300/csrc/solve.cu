// Solve path: CSR SpMV, restriction, batched local solves, prolongation,
// coarse correction and preconditioned CG, all on one stream.
//
// Preconditioner (Sec. 2, eq. "AS2"; closed form at the end of Sec. 3.2):
//   y0 = Z E^-1 Z^T r ;  s = r - A y0 ;  w = sum_i R_i^T A_i^-1 R_i s ;
//   z  = y0 + w - Z E^-1 Z^T (A w).
// PCG: A is SPD (Sec. 2) and M^-1_AS,2 symmetric (eq. "AS2").
#include <chrono>

#include "setup.hpp"

namespace geneo {

// y = A x; 8 lanes per row
__global__ void k_spmv(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                       const double *__restrict__ val, const double *__restrict__ x,
                       double *__restrict__ y, int64_t n) {
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gt >> 3;
  const int lane = threadIdx.x & 7;
  double s = 0;
  if (row < n)
    for (int32_t k = rowptr[row] + lane; k < rowptr[row + 1]; k += 8) s = fma(val[k], x[col[k]], s);
  s += __shfl_xor_sync(0xffffffffu, s, 4);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  if (row < n && lane == 0) y[row] = s;
}

// y = b - A x
__global__ void k_residual(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                           const double *__restrict__ val, const double *__restrict__ x,
                           const double *__restrict__ b, double *__restrict__ y, int64_t n) {
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gt >> 3;
  const int lane = threadIdx.x & 7;
  double s = 0;
  if (row < n)
    for (int32_t k = rowptr[row] + lane; k < rowptr[row + 1]; k += 8) s = fma(val[k], x[col[k]], s);
  s += __shfl_xor_sync(0xffffffffu, s, 4);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  if (row < n && lane == 0) y[row] = b[row] - s;
}

// padded local vector x_loc[p] = s[l2g[p]] (0 on padding)
__global__ void k_restrict(const int32_t *__restrict__ l2g, const double *__restrict__ s,
                           double *__restrict__ xl, int64_t len) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= len) return;
  const int32_t g = l2g[p];
  xl[p] = g >= 0 ? s[g] : 0.0;
}

// w[e] = sum over the local slots holding e (deterministic gather-sum)
__global__ void k_prolong(const int64_t *__restrict__ ptr, const int64_t *__restrict__ slot,
                          const double *__restrict__ yl, double *__restrict__ w, int64_t n) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  double s = 0;
  for (int64_t k = ptr[e]; k < ptr[e + 1]; ++k) s += yl[slot[k]];
  w[e] = s;
}

// t[a] = (Z^T r)_a, one column per warp (CSC): split near-kernel columns
// have a few entries, GenEO columns one per dof of their subdomain
__global__ void k_zt(const int64_t *__restrict__ zptr, const int32_t *__restrict__ zrow,
                     const double *__restrict__ zval, const double *__restrict__ r,
                     double *__restrict__ t, int64_t n0) {
  const int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int l = threadIdx.x & 31;
  if (a >= n0) return;
  double s = 0;
  for (int64_t k = zptr[a] + l; k < zptr[a + 1]; k += 32) s = fma(zval[k], r[zrow[k]], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (l == 0) t[a] = s;
}

// y[e] = (Z u)_e, one row per thread (CSR)
__global__ void k_z(const int64_t *__restrict__ zptr, const int32_t *__restrict__ zcol,
                    const double *__restrict__ zval, const double *__restrict__ u,
                    double *__restrict__ y, int64_t n) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  double s = 0;
  for (int64_t k = zptr[e]; k < zptr[e + 1]; ++k) s = fma(zval[k], u[zcol[k]], s);
  y[e] = s;
}

// z = y0 + w - c
__global__ void k_combine(const double *__restrict__ y0, const double *__restrict__ w,
                          const double *__restrict__ c, double *__restrict__ z, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) z[i] = (y0[i] + w[i]) - c[i];
}

// ---------------------------------------------------------------------------
// deterministic dot products: fixed grid, block partials, one final block

constexpr int kDotBlocks = 512;

__global__ void k_dot_partial(const double *__restrict__ a, const double *__restrict__ b, int64_t n,
                              double *__restrict__ part) {
  __shared__ double sh[256];
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

__global__ void k_dot_final(const double *__restrict__ part, int np, double *__restrict__ out) {
  __shared__ double sh[32];
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
                cudaStream_t s) {
  c->launches += 2;
  k_dot_partial<<<kDotBlocks, 256, 0, s>>>(a, b, n, c->partials.p);
  k_dot_final<<<1, 256, 0, s>>>(c->partials.p, kDotBlocks, out);
}

// scalars: 0 rz, 1 pq, 2 rr, 3 rz_new, 4 bb
// x += alpha p ; r -= alpha q  with alpha = rz / pq
__global__ void k_update_xr(const double *__restrict__ sc, const double *__restrict__ p,
                            const double *__restrict__ q, double *__restrict__ x,
                            double *__restrict__ r, int64_t n) {
  const double alpha = sc[0] / sc[1];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, q[i], r[i]);
  }
}

// p = z + beta p with beta = rz_new / rz; then rz = rz_new
__global__ void k_update_p(double *__restrict__ sc, const double *__restrict__ z,
                           double *__restrict__ p, int64_t n) {
  const double beta = sc[3] / sc[0];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = fma(beta, p[i], z[i]);
}

__global__ void k_shift_rz(double *sc) { sc[0] = sc[3]; }

__global__ void k_copy(const double *__restrict__ a, double *__restrict__ b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

// ---------------------------------------------------------------------------

void spmv(geneo_ctx *c, const double *x, double *y, cudaStream_t s) {
  const int64_t n = c->topo.ndofs();
  c->launches += 1;
  k_spmv<<<grid_for(n * 8, 256), 256, 0, s>>>(c->d_rowptr.p, c->d_col.p, c->d_val.p, x, y, n);
  GENEO_CHECK_LAUNCH();
}

void local_solve(geneo_ctx *c, const double *r, double *w, cudaStream_t s) {
  const int64_t n = c->topo.ndofs();
  c->launches += 4;
  k_restrict<<<grid_for(c->loc.vlen, 256), 256, 0, s>>>(c->d_l2g.p, r, c->loc_x.p, c->loc.vlen);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->prof) {
    e0 = c->ev_take();
    e1 = c->ev_take();
    c->ev_local.push_back({e0, e1});
  }
  if (c->local_prec == GENEO_PREC_FP32) {
    // split inverse: float32 C_j r_j plus the float64 gradient part
    symv_batch<float>(c->loc, c->loc_f32.p, c->loc_x.p, c->loc_y.p, c->d_err.p, s, e0, e1);
    split_gradient_apply(c, c->loc_x.p, c->loc_y.p, s);
    c->launches += 4;
  } else {
    symv_batch<double>(c->loc, c->loc_f64.p, c->loc_x.p, c->loc_y.p, c->d_err.p, s, e0, e1);
  }
  k_prolong<<<grid_for(n, 256), 256, 0, s>>>(c->d_g2l_ptr.p, c->d_g2l.p, c->loc_y.p, w, n);
  GENEO_CHECK_LAUNCH();
}

void coarse_solve(geneo_ctx *c, const double *r, double *y, cudaStream_t s) {
  const int64_t n = c->topo.ndofs();
  if (c->n0 == 0) {
    GENEO_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * n, s));
    return;
  }
  if (c->mf) {
    c->launches += 2 + mf_launches_per_solve(c);
    k_zt<<<grid_for(c->n0 * 32, 256), 256, 0, s>>>(c->d_zc_ptr.p, c->d_zc_row.p, c->d_zc_val.p, r,
                                              c->crs_x.p, c->n0);
    if (c->prof) {
      cudaEvent_t e0 = c->ev_take(), e1 = c->ev_take();
      c->ev_coarse.push_back({e0, e1});
      record_event(e0, s);
      mf_solve(c, c->crs_x.p, c->crs_y.p, s);
      record_event(e1, s);
    } else {
      mf_solve(c, c->crs_x.p, c->crs_y.p, s);
    }
    k_z<<<grid_for(n, 256), 256, 0, s>>>(c->d_zr_ptr.p, c->d_zr_col.p, c->d_zr_val.p, c->crs_y.p,
                                         y, n);
    GENEO_CHECK_LAUNCH();
    return;
  }
  c->launches += 4;
  k_zt<<<grid_for(c->n0 * 32, 256), 256, 0, s>>>(c->d_zc_ptr.p, c->d_zc_row.p, c->d_zc_val.p, r,
                                            c->crs_x.p, c->n0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->prof) {
    e0 = c->ev_take();
    e1 = c->ev_take();
    c->ev_coarse.push_back({e0, e1});
  }
  symv_batch<double>(c->crs, c->crs_f64.p, c->crs_x.p, c->crs_y.p, c->d_err.p, s, e0, e1);
  k_z<<<grid_for(n, 256), 256, 0, s>>>(c->d_zr_ptr.p, c->d_zr_col.p, c->d_zr_val.p, c->crs_y.p,
                                       y, n);
  GENEO_CHECK_LAUNCH();
}

void apply_preconditioner(geneo_ctx *c, const double *r, double *z, cudaStream_t s) {
  const int64_t n = c->topo.ndofs();
  if (c->n0 == 0) {
    local_solve(c, r, z, s);
    return;
  }
  c->launches += 2;
  coarse_solve(c, r, c->v_y0.p, s);
  k_residual<<<grid_for(n * 8, 256), 256, 0, s>>>(c->d_rowptr.p, c->d_col.p, c->d_val.p,
                                                  c->v_y0.p, r, c->v_s.p, n);
  local_solve(c, c->v_s.p, c->v_w.p, s);
  spmv(c, c->v_w.p, c->v_t.p, s);
  coarse_solve(c, c->v_t.p, c->v_c.p, s);
  k_combine<<<grid_for(n, 256), 256, 0, s>>>(c->v_y0.p, c->v_w.p, c->v_c.p, z, n);
  GENEO_CHECK_LAUNCH();
}

// second half of a PCG iteration: z = M^-1 r, rz_new = (r, z), p = z + beta p
static void pcg_precond_half(geneo_ctx *c, cudaStream_t s) {
  const int64_t n = c->topo.ndofs();
  double *sc = c->scal.p;
  apply_preconditioner(c, c->p_r.p, c->p_z.p, s);
  dot(c, c->p_r.p, c->p_z.p, n, sc + 3, s);
  c->launches += 2;
  k_update_p<<<grid_for(n, 256), 256, 0, s>>>(sc, c->p_z.p, c->p_p.p, n);
  k_shift_rz<<<1, 1, 0, s>>>(sc);
  GENEO_CHECK_LAUNCH();
}

// first half: q = A p, alpha = rz / (p, q), x += alpha p, r -= alpha q,
// rr = (r, r), scalars copied to the pinned host mirror
static void pcg_step_half(geneo_ctx *c, double *x, cudaStream_t s) {
  const int64_t n = c->topo.ndofs();
  double *sc = c->scal.p;
  spmv(c, c->p_p.p, c->p_q.p, s);
  dot(c, c->p_p.p, c->p_q.p, n, sc + 1, s);
  c->launches += 1;
  k_update_xr<<<grid_for(n, 256), 256, 0, s>>>(sc, c->p_p.p, c->p_q.p, x, c->p_r.p, n);
  dot(c, c->p_r.p, c->p_r.p, n, sc + 2, s);
  GENEO_CUDA(cudaMemcpyAsync(c->h_scal, sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  GENEO_CHECK_LAUNCH();
}

// Captures [second half ; first half] of an iteration on the context's
// capture stream, with x = p_x; replayed on the caller's stream for every
// iteration after the first.
static void ensure_pcg_graph(geneo_ctx *c) {
  const int key = c->local_prec * 2 + (c->prof ? 1 : 0);
  if (c->pcg_exec && c->pcg_key == key) return;
  c->drop_graph();
  const int64_t l0 = c->launches;
  const size_t nl = c->ev_local.size(), nc = c->ev_coarse.size();
  cudaStream_t cs = c->cap_stream;
  GENEO_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaGraph_t graph = nullptr;
  try {
    pcg_precond_half(c, cs);
    pcg_step_half(c, c->p_x.p, cs);
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

int pcg(geneo_ctx *c, const double *b, double *x, double tol, int maxit, geneo_solve_info *info,
        cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t n = c->topo.ndofs();
  double *sc = c->scal.p;
  double *hs = c->h_scal;
  const unsigned g = grid_for(n, 256);
  const bool graph = c->opt.use_graph != 0;
  double *xw = graph ? c->p_x.p : x;  // the graph is built on the context's own x
  GENEO_CUDA(cudaMemsetAsync(xw, 0, sizeof(double) * n, s));
  c->launches += 2;
  k_copy<<<g, 256, 0, s>>>(b, c->p_r.p, n);
  dot(c, b, b, n, sc + 4, s);
  apply_preconditioner(c, c->p_r.p, c->p_z.p, s);
  k_copy<<<g, 256, 0, s>>>(c->p_z.p, c->p_p.p, n);
  dot(c, c->p_r.p, c->p_z.p, n, sc + 0, s);
  GENEO_CUDA(cudaMemcpyAsync(hs, sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  GENEO_CUDA(cudaStreamSynchronize(s));
  const double bnorm = std::sqrt(hs[4]);
  int status = GENEO_NOT_CONVERGED, it = 0;
  double rel = 1.0;
  if (bnorm == 0.0) {
    status = GENEO_OK;
    rel = 0.0;
  } else {
    for (it = 1; it <= maxit; ++it) {
      const bool replay = graph && it > 1;
      if (it == 1) {
        pcg_step_half(c, xw, s);
      } else if (replay) {
        ensure_pcg_graph(c);
        GENEO_CUDA(cudaGraphLaunch(c->pcg_exec, s));
        c->launches += c->pcg_graph_launches;
      } else {
        pcg_precond_half(c, s);
        pcg_step_half(c, xw, s);
      }
      GENEO_CUDA(cudaStreamSynchronize(s));
      if (replay && c->prof) harvest_graph_events(c);
      if (!(hs[1] > 0.0) || !std::isfinite(hs[1]) || !std::isfinite(hs[2])) {
        status = GENEO_ERR_BREAKDOWN;
        break;
      }
      rel = std::sqrt(hs[2]) / bnorm;
      if (rel <= tol) {
        status = GENEO_OK;
        break;
      }
    }
    if (it > maxit) it = maxit;
  }
  if (xw != x) {
    c->launches += 1;
    k_copy<<<g, 256, 0, s>>>(xw, x, n);
    GENEO_CHECK_LAUNCH();
  }
  GENEO_CUDA(cudaStreamSynchronize(s));
  check_device_error(c, s);
  if (info) {
    info->iters = it;
    info->relres = rel;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return status;
}

}  // namespace geneo
