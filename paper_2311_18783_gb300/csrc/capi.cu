// C-ABI entry points (include/geneo.h): argument checks, status codes and
// the thread-local error message.  No exception crosses this boundary.
#include <cstring>
#include <string>

#include "compose.hpp"
#include "setup.hpp"

namespace {
thread_local std::string g_last_error;

int fail(int status, const std::string &msg) {
  g_last_error = msg;
  return status;
}

template <class F>
int guarded(F &&f) {
  try {
    return f();
  } catch (const geneo::Error &e) {
    return fail(e.status, e.what());
  } catch (const std::bad_alloc &) {
    return fail(GENEO_ERR_OOM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(GENEO_ERR_CUDA, e.what());
  } catch (...) {
    return fail(GENEO_ERR_CUDA, "unknown failure");
  }
}

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }
constexpr int kMaxRhs = 16;
}  // namespace

void geneo_ctx::drop_graph() {
  if (pcg_exec) cudaGraphExecDestroy(pcg_exec);
  pcg_exec = nullptr;
  pcg_key = -1;
  if (seg_exec) cudaGraphExecDestroy(seg_exec);
  seg_exec = nullptr;
  seg_key = -1;
  for (auto &p : g_ev_local) ev_free.insert(ev_free.end(), {p.first, p.second});
  for (auto &p : g_ev_coarse) ev_free.insert(ev_free.end(), {p.first, p.second});
  g_ev_local.clear();
  g_ev_coarse.clear();
}

geneo_ctx::~geneo_ctx() {
  drop_graph();
  if (cap_stream) cudaStreamDestroy(cap_stream);
  for (auto &p : ev_local) ev_free.insert(ev_free.end(), {p.first, p.second});
  for (auto &p : ev_coarse) ev_free.insert(ev_free.end(), {p.first, p.second});
  for (cudaEvent_t e : ev_free) cudaEventDestroy(e);
  if (h_scal) cudaFreeHost(h_scal);
  if (h_seg) cudaFreeHost(h_seg);
  if (h_act) cudaFreeHost(h_act);
  if (stream) cudaStreamDestroy(stream);
}

cudaEvent_t geneo_ctx::ev_take() {
  if (ev_free.empty()) {
    cudaEvent_t e;
    GENEO_CUDA(cudaEventCreate(&e));
    return e;
  }
  cudaEvent_t e = ev_free.back();
  ev_free.pop_back();
  return e;
}

extern "C" {

void geneo_default_options(geneo_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = GENEO_PREC_FP64;
  o->coarse = GENEO_COARSE_SNK;
  o->geneo = 1;
  o->tau_convention = GENEO_TAU_RECIPROCAL;
  o->lobpcg_block = 8;
  o->lobpcg_maxit = 200;
  o->lobpcg_tol = 1e-8;
  o->seed = 1;
  o->use_graph = 1;
}

// Argument checks shared by geneo_setup and geneo_setup_topology; fills o.
static int check_setup_args(const geneo_problem *p, const geneo_options *opt, geneo_ctx **out,
                            geneo_options &o) {
  if (!p || !out) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || !(p->hx > 0) || !(p->hy > 0) || !(p->hz > 0))
    return fail(GENEO_ERR_INVALID_ARG, "grid sizes must be positive");
  if (!p->active || !p->mu_inv || !p->eps) return fail(GENEO_ERR_INVALID_ARG, "null array");
  if (!(p->gamma > 0)) return fail(GENEO_ERR_INVALID_ARG, "gamma must be > 0");
  if (p->overlap < 1) return fail(GENEO_ERR_INVALID_ARG, "overlap must be >= 1");
  if (!p->cell_part &&
      (p->px < 1 || p->py < 1 || p->pz < 1 || p->px > p->nx || p->py > p->ny || p->pz > p->nz))
    return fail(GENEO_ERR_INVALID_ARG, "box counts must lie in [1, cells per axis]");
  if (!(p->tau > 0)) return fail(GENEO_ERR_INVALID_ARG, "tau must be > 0");
  const int64_t nc = (int64_t)p->nx * p->ny * p->nz;
  if (nc > (int64_t)1 << 28) return fail(GENEO_ERR_INVALID_ARG, "mesh too large for int32 indices");
  for (int64_t c = 0; c < nc; ++c)
    if (p->active[c] && (!(p->mu_inv[c] > 0) || !(p->eps[c] > 0)))
      return fail(GENEO_ERR_INVALID_ARG, "mu^-1 and eps must be > 0 on active cells");
  if (p->cell_part)
    for (int64_t c = 0; c < nc; ++c)
      if (p->active[c] && (p->cell_part[c] < 0 || p->cell_part[c] >= (1 << 24)))
        return fail(GENEO_ERR_INVALID_ARG, "cell_part must lie in [0, 2^24) on active cells");
  geneo_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != GENEO_PREC_FP64 && o.precision != GENEO_PREC_FP32 &&
      o.precision != GENEO_PREC_BF16)
    return fail(GENEO_ERR_INVALID_ARG, "unknown precision");
  if (o.coarse != GENEO_COARSE_NONE && o.coarse != GENEO_COARSE_SNK &&
      o.coarse != GENEO_COARSE_NK)
    return fail(GENEO_ERR_INVALID_ARG, "unknown coarse mode");
  if (o.lobpcg_block < 1 || o.lobpcg_block > 16 || o.lobpcg_maxit < 1 || !(o.lobpcg_tol > 0))
    return fail(GENEO_ERR_INVALID_ARG, "bad LOBPCG parameters");
  if (o.warm_start && o.lobpcg_block != 8)
    return fail(GENEO_ERR_INVALID_ARG, "a warm start needs lobpcg_block = 8");
  if (o.keep_eigvecs != 0 && o.keep_eigvecs != 1)
    return fail(GENEO_ERR_INVALID_ARG, "keep_eigvecs must be 0 or 1");
  if (o.lobpcg_neumann != 0 && o.lobpcg_neumann != 1)
    return fail(GENEO_ERR_INVALID_ARG, "lobpcg_neumann must be 0 or 1");
  if (o.balanced != 0 && o.balanced != 1)
    return fail(GENEO_ERR_INVALID_ARG, "balanced must be 0 or 1");
  if (o.geneo_pencil != GENEO_PENCIL_FILTERED && o.geneo_pencil != GENEO_PENCIL_CLASSICAL)
    return fail(GENEO_ERR_INVALID_ARG, "unknown GenEO pencil");
  if (o.autotune != 0 && o.autotune != 1)
    return fail(GENEO_ERR_INVALID_ARG, "autotune must be 0 or 1");
  if ((o.coarse_dense != 0 && o.coarse_dense != 1) || o.coarse_leaf < 0 ||
      (o.use_graph != 0 && o.use_graph != 1) || (o.gradient_shift != 0 && o.gradient_shift != 1))
    return fail(GENEO_ERR_INVALID_ARG, "bad coarse factor or graph options");
  return GENEO_OK;
}

// A context holding the problem copy (no device work yet).
static geneo_ctx *new_context(const geneo_problem *p, const geneo_options &o) {
  const int64_t nc = (int64_t)p->nx * p->ny * p->nz;
  auto c = new geneo_ctx();
  c->nx = p->nx;
  c->ny = p->ny;
  c->nz = p->nz;
  c->h[0] = p->hx;
  c->h[1] = p->hy;
  c->h[2] = p->hz;
  c->gamma = p->gamma;
  c->tau = p->tau;
  c->tau_p = o.tau_convention == GENEO_TAU_PAPER ? p->tau : 1.0 / p->tau;
  c->px = p->px;
  c->py = p->py;
  c->pz = p->pz;
  c->overlap = p->overlap;
  c->active.assign(p->active, p->active + nc);
  c->mu_inv.assign(p->mu_inv, p->mu_inv + nc);
  c->eps.assign(p->eps, p->eps + nc);
  if (p->cell_part) c->cell_part.assign(p->cell_part, p->cell_part + nc);
  if (p->natural_faces) c->natural.assign(p->natural_faces, p->natural_faces + nc);
  c->opt = o;
  c->balanced = o.balanced != 0;
  return c;
}

int geneo_setup(const geneo_problem *p, const geneo_options *opt, geneo_ctx **out) {
  geneo_options o;
  const int rc = check_setup_args(p, opt, out, o);
  if (rc != GENEO_OK) return rc;
  return guarded([&]() {
    geneo_ctx *c = new_context(p, o);
    try {
      GENEO_CUDA(cudaGetDevice(&c->device));
      c->sm_count = geneo::device_sm_count();
      GENEO_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      GENEO_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
      geneo::setup_all(c);
    } catch (...) {
      delete c;
      throw;
    }
    *out = c;
    return GENEO_OK;
  });
}

int geneo_setup_topology(const geneo_problem *p, const geneo_options *opt, geneo_ctx **out) {
  geneo_options o;
  const int rc = check_setup_args(p, opt, out, o);
  if (rc != GENEO_OK) return rc;
  return guarded([&]() {
    geneo_ctx *c = new_context(p, o);
    c->host_only = true;
    try {
      geneo::setup_topology(c);
    } catch (...) {
      delete c;
      throw;
    }
    *out = c;
    return GENEO_OK;
  });
}

void geneo_destroy(geneo_ctx *c) {
  if (!c) return;
  if (!c->host_only) cudaDeviceSynchronize();
  delete c;
}

int geneo_query(const geneo_ctx *c, geneo_sizes *o) {
  if (!c || !o) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  std::memset(o, 0, sizeof(*o));
  o->nverts = c->topo.nverts;
  o->ncells = c->topo.ncells;
  o->ntets = c->topo.ntets();
  o->nedges = c->topo.nedges();
  o->n = c->topo.ndofs();
  o->nnz = c->topo.nnz();
  o->nsub = c->dec.nsub;
  o->k0 = c->dec.k0;
  o->k1 = c->dec.k1;
  o->sum_ni = c->dec.N_off.empty() ? 0 : c->dec.N_off.back();
  for (int i = 0; i < c->dec.nsub; ++i) o->max_ni = std::max<int64_t>(o->max_ni, c->dec.ni(i));
  o->n0 = c->n0;
  o->n0_snk = c->n0_snk;
  o->n0_geneo = c->n0_geneo;
  o->local_factor_bytes = c->loc_f64.bytes() + c->loc_f32.bytes() + geneo::tc_factor_bytes(c);
  o->coarse_factor_bytes = c->mf ? geneo::mf_factor_bytes(c) : c->crs_f64.bytes();
  o->setup_seconds = c->setup_seconds;
  return GENEO_OK;
}

int geneo_assemble_rhs(geneo_ctx *c, const double *f, double *b, void *s) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c || !f || !b) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  return guarded([&]() {
    geneo::assemble_rhs(c, f, b, as_stream(s));
    return GENEO_OK;
  });
}

int geneo_spmv(geneo_ctx *c, const double *x, double *y, void *s) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c || !x || !y) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  return guarded([&]() {
    geneo::spmv(c, x, y, as_stream(s));
    return GENEO_OK;
  });
}

int geneo_local_solve(geneo_ctx *c, const double *r, double *w, void *s) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c || !r || !w) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  return guarded([&]() {
    geneo::local_solve(c, r, w, as_stream(s));
    return GENEO_OK;
  });
}

int geneo_coarse_solve(geneo_ctx *c, const double *r, double *y, void *s) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c || !r || !y) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  return guarded([&]() {
    geneo::coarse_solve(c, r, y, as_stream(s));
    return GENEO_OK;
  });
}

int geneo_apply_preconditioner(geneo_ctx *c, const double *r, double *z, void *s) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c || !r || !z) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  return guarded([&]() {
    geneo::apply_preconditioner(c, r, z, as_stream(s));
    return GENEO_OK;
  });
}

int geneo_solve(geneo_ctx *c, const double *b, double *x, double tol, int32_t maxit,
                geneo_solve_info *info, void *s) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c || !b || !x) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  if (!(tol > 0) || maxit < 1) return fail(GENEO_ERR_INVALID_ARG, "tol must be > 0, maxit >= 1");
  return guarded([&]() { return geneo::pcg(c, b, x, tol, maxit, info, as_stream(s)); });
}

int geneo_solve_refined(geneo_ctx *c, const double *b, double *x, double tol, int32_t maxit,
                        int32_t nref, geneo_solve_info *info, void *s) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c || !b || !x) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  if (!(tol > 0) || maxit < 1) return fail(GENEO_ERR_INVALID_ARG, "tol must be > 0, maxit >= 1");
  if (nref < 0 || nref > 16) return fail(GENEO_ERR_INVALID_ARG, "nref must be in 0..16");
  if (b == x) return fail(GENEO_ERR_INVALID_ARG, "b and x must not alias");
  return guarded([&]() { return geneo::pcg_refined(c, b, x, tol, maxit, nref, info, as_stream(s)); });
}

int geneo_solve_gmres(geneo_ctx *c, const double *b, double *x, double tol, int32_t maxit,
                      int32_t restart, geneo_solve_info *info, void *s) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c || !b || !x) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  if (!(tol > 0) || maxit < 1) return fail(GENEO_ERR_INVALID_ARG, "tol must be > 0, maxit >= 1");
  if (restart < 1 || restart > 1000) return fail(GENEO_ERR_INVALID_ARG, "restart must be in 1..1000");
  if (b == x) return fail(GENEO_ERR_INVALID_ARG, "b and x must not alias");
  return guarded([&]() { return geneo::gmres(c, b, x, tol, maxit, restart, info, as_stream(s)); });
}

int geneo_symv_config_count(int32_t precision) {
  if (precision == GENEO_PREC_FP32) return geneo::symv_candidates<float>();
  if (precision == GENEO_PREC_FP64) return geneo::symv_candidates<double>();
  return fail(GENEO_ERR_INVALID_ARG, "precision must be FP32 or FP64");
}

int geneo_use_symv_config(geneo_ctx *c, int32_t precision, int32_t index) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  const int n = geneo_symv_config_count(precision);
  if (n < 0) return n;
  if (index < 0 || index >= n) return fail(GENEO_ERR_INVALID_ARG, "configuration index out of range");
  c->loc.symv_cfg[precision == GENEO_PREC_FP64 ? 1 : 0] = index;
  return GENEO_OK;
}

int geneo_use_gradient_precision(geneo_ctx *c, int32_t precision) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  if (precision == GENEO_PREC_FP64) {
    c->grad32 = false;
    return GENEO_OK;
  }
  if (precision != GENEO_PREC_FP32) return fail(GENEO_ERR_INVALID_ARG, "precision must be FP32 or FP64");
  if (!c->xi || !c->xi->s_inv32.p)
    return fail(GENEO_ERR_STATE, "the split factors (options.precision FP32 or BF16) were not built");
  c->grad32 = true;
  return GENEO_OK;
}

int geneo_use_balanced(geneo_ctx *c, int32_t on) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  if (on != 0 && on != 1) return fail(GENEO_ERR_INVALID_ARG, "on must be 0 or 1");
  c->balanced = on != 0;
  return GENEO_OK;
}

int geneo_use_persistent_coarse(geneo_ctx *c, int32_t on) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  if (on != 0 && on != 1) return fail(GENEO_ERR_INVALID_ARG, "on must be 0 or 1");
  c->mf_persist = on != 0;
  return GENEO_OK;
}

int geneo_apply_preconditioner_block(geneo_ctx *c, const double *r, double *z, int32_t nrhs,
                                     void *s) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c || !r || !z) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  if (nrhs < 1 || nrhs > kMaxRhs) return fail(GENEO_ERR_INVALID_ARG, "nrhs must be in 1..16");
  return guarded([&]() {
    geneo::reserve_rhs(c, nrhs);
    geneo::apply_preconditioner(c, r, z, as_stream(s), nrhs);
    return GENEO_OK;
  });
}

int geneo_solve_block(geneo_ctx *c, const double *b, double *x, int32_t nrhs, double tol,
                      int32_t maxit, geneo_solve_info *info, void *s) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c || !b || !x) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  if (nrhs < 1 || nrhs > kMaxRhs) return fail(GENEO_ERR_INVALID_ARG, "nrhs must be in 1..16");
  if (!(tol > 0) || maxit < 1) return fail(GENEO_ERR_INVALID_ARG, "tol must be > 0, maxit >= 1");
  return guarded(
      [&]() { return geneo::pcg(c, b, x, tol, maxit, info, as_stream(s), nrhs); });
}

int geneo_solve_segments(geneo_ctx *c, const double *b, double *x, double tol, int32_t maxit,
                         geneo_solve_info *info, void *s) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c || !b || !x) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  if (!(tol > 0) || maxit < 1) return fail(GENEO_ERR_INVALID_ARG, "tol must be > 0, maxit >= 1");
  return guarded([&]() { return geneo::pcg_segments(c, b, x, tol, maxit, info, as_stream(s)); });
}

int geneo_compose_size(int32_t nprob, const geneo_problem *probs, int32_t *dims, double *h) {
  if (!dims || !h) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  return guarded([&]() {
    geneo::Composite c;
    geneo::compose_problems(nprob, probs, false, c);
    dims[0] = c.nx;
    dims[1] = c.ny;
    dims[2] = c.nz;
    *h = c.h;
    return GENEO_OK;
  });
}

int geneo_compose(int32_t nprob, const geneo_problem *probs, uint8_t *active, double *mu_inv,
                  double *eps, int32_t *cell_part, int32_t *zoff) {
  if (!active || !mu_inv || !eps || !cell_part) return fail(GENEO_ERR_INVALID_ARG, "null array");
  return guarded([&]() {
    geneo::Composite c;
    geneo::compose_problems(nprob, probs, true, c);
    std::memcpy(active, c.active.data(), c.active.size());
    std::memcpy(mu_inv, c.mu_inv.data(), sizeof(double) * c.mu_inv.size());
    std::memcpy(eps, c.eps.data(), sizeof(double) * c.eps.size());
    std::memcpy(cell_part, c.part.data(), sizeof(int32_t) * c.part.size());
    if (zoff) std::memcpy(zoff, c.zoff.data(), sizeof(int32_t) * c.zoff.size());
    return GENEO_OK;
  });
}

int geneo_compose_field(int32_t nprob, const geneo_problem *probs, const double *const *f_slot,
                        int32_t nrhs, double *f_out) {
  return guarded([&]() {
    geneo::Composite c;
    geneo::compose_problems(nprob, probs, false, c);
    geneo::compose_field(nprob, probs, c, f_slot, nrhs, f_out);
    return GENEO_OK;
  });
}

int geneo_setup_batch(int32_t nprob, const geneo_problem *probs, const geneo_options *opt,
                      geneo_ctx **out) {
  if (!out) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  geneo::Composite c;
  const int rc = guarded([&]() {
    geneo::compose_problems(nprob, probs, true, c);
    return GENEO_OK;
  });
  if (rc != GENEO_OK) return rc;
  geneo_problem q{};
  q.nx = c.nx;
  q.ny = c.ny;
  q.nz = c.nz;
  q.hx = q.hy = q.hz = c.h;
  q.active = c.active.data();
  q.mu_inv = c.mu_inv.data();
  q.eps = c.eps.data();
  q.gamma = 1.0;
  q.px = q.py = q.pz = 1;
  q.overlap = probs[0].overlap;
  q.tau = probs[0].tau;
  q.cell_part = c.part.data();
  return geneo_setup(&q, opt, out);
}

int geneo_solve_host(geneo_ctx *c, const double *bh, double *xh, double tol, int32_t maxit,
                     geneo_solve_info *info, void *s) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c || !bh || !xh) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  if (!(tol > 0) || maxit < 1) return fail(GENEO_ERR_INVALID_ARG, "tol must be > 0, maxit >= 1");
  return guarded([&]() {
    cudaStream_t st = as_stream(s);
    const int64_t n = c->topo.ndofs();
    // b and x live in two vectors the context reserves for this call
    GENEO_CUDA(cudaMemcpyAsync(c->h_b.p, bh, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    const int rc = geneo::pcg(c, c->h_b.p, c->h_x.p, tol, maxit, info, st);
    GENEO_CUDA(cudaMemcpyAsync(xh, c->h_x.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    GENEO_CUDA(cudaStreamSynchronize(st));
    return rc;
  });
}

int geneo_use_precision(geneo_ctx *c, int32_t precision) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  if (precision == GENEO_PREC_FP64 && c->loc_f64.p) {
    c->local_prec = GENEO_PREC_FP64;
    return GENEO_OK;
  }
  if (precision == GENEO_PREC_FP32 && c->loc_f32.p) {
    c->local_prec = GENEO_PREC_FP32;
    return GENEO_OK;
  }
  if (precision == GENEO_PREC_BF16 && c->tc) {
    c->local_prec = GENEO_PREC_BF16;
    return GENEO_OK;
  }
  return fail(GENEO_ERR_STATE, "the requested local factors were not built");
}

int geneo_profile_enable(geneo_ctx *c, int32_t on) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  c->prof = on != 0;
  return GENEO_OK;
}

int geneo_profile_read(geneo_ctx *c, geneo_profile *o) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!c || !o) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  return guarded([&]() {
    std::memset(o, 0, sizeof(*o));
    o->launches = c->launches;
    auto sum = [&](std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &v, double &ms) {
      for (auto &p : v) {
        GENEO_CUDA(cudaEventSynchronize(p.second));
        float t = 0;
        GENEO_CUDA(cudaEventElapsedTime(&t, p.first, p.second));
        ms += t;
        c->ev_free.push_back(p.first);
        c->ev_free.push_back(p.second);
      }
      const int64_t k = (int64_t)v.size();
      v.clear();
      return k;
    };
    o->local_symv_launches = sum(c->ev_local, o->local_symv_ms) + c->acc_local_n;
    o->coarse_symv_launches = sum(c->ev_coarse, o->coarse_symv_ms) + c->acc_coarse_n;
    o->local_symv_ms += c->acc_local_ms;
    o->coarse_symv_ms += c->acc_coarse_ms;
    c->acc_local_ms = c->acc_coarse_ms = 0;
    c->acc_local_n = c->acc_coarse_n = 0;
    o->local_symv_bytes = c->local_prec == GENEO_PREC_BF16
                              ? geneo::tc_factor_bytes(c)
                              : c->loc.ntiles * (int64_t)geneo::kTileElems *
                                    (c->local_prec == GENEO_PREC_FP32 ? (int64_t)sizeof(float)
                                                                      : (int64_t)sizeof(double));
    o->coarse_solve_bytes = geneo::mf_solve_bytes(c);
    int64_t fl = 0;
    for (int i = 0; i < c->dec.nsub; ++i) fl += 2 * c->dec.ni(i) * c->dec.ni(i);
    o->local_symv_flops = fl;
    c->launches = 0;
    return GENEO_OK;
  });
}

int geneo_export(const geneo_ctx *c, const char *name, void *dst, int64_t cap, int64_t *size) {
  if (!c || !name) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  return guarded([&]() -> int {
    std::vector<unsigned char> buf;
    auto put = [&](const void *p, size_t bytes) {
      buf.assign((const unsigned char *)p, (const unsigned char *)p + bytes);
    };
    const std::string nm(name);
    if (c->host_only && (nm == "A_val" || nm == "loc_f32" || nm == "mlp_features" || nm == "eig_V"))
      return fail(GENEO_ERR_STATE, "topology-only context: no device data");
    const geneo::Topology &t = c->topo;
    if (nm == "edges") put(t.edges.data(), t.edges.size() * 4);
    else if (nm == "dir_edge") put(t.dir_edge.data(), t.dir_edge.size());
    else if (nm == "dof_edge") put(t.dof_edge.data(), t.dof_edge.size() * 4);
    else if (nm == "dof_vert") put(t.dof_vert.data(), t.dof_vert.size() * 4);
    else if (nm == "A_rowptr") put(t.rowptr.data(), t.rowptr.size() * 4);
    else if (nm == "A_col") put(t.col.data(), t.col.size() * 4);
    else if (nm == "A_val") {
      auto v = c->d_val.download(c->stream);
      put(v.data(), v.size() * 8);
    } else if (nm == "N_off") put(c->dec.N_off.data(), c->dec.N_off.size() * 8);
    else if (nm == "N_idx") put(c->dec.N_idx.data(), c->dec.N_idx.size() * 4);
    else if (nm == "owner") put(c->dec.owner.data(), c->dec.owner.size() * 4);
    else if (nm == "snk_sub") put(c->snk.sub.data(), c->snk.sub.size() * 4);
    else if (nm == "snk_vert") put(c->snk.vert.data(), c->snk.vert.size() * 4);
    else if (nm == "geneo_sub") put(c->geneo_sub.data(), c->geneo_sub.size() * 4);
    else if (nm == "geneo_lambda") put(c->geneo_lambda.data(), c->geneo_lambda.size() * 8);
    else if (nm == "geneo_found") put(c->geneo_found.data(), c->geneo_found.size() * 4);
    else if (nm == "Zcol_ptr") put(c->zc_ptr.data(), c->zc_ptr.size() * 8);
    else if (nm == "Zcol_row") put(c->zc_row.data(), c->zc_row.size() * 4);
    else if (nm == "Zcol_val") put(c->zc_val.data(), c->zc_val.size() * 8);
    else if (nm == "loc_f32") {
      auto v = c->loc_f32.download(c->stream);
      put(v.data(), v.size() * 4);
    } else if (nm == "loc_nt") put(c->loc.nt.data(), c->loc.nt.size() * 4);
    else if (nm == "loc_toff") put(c->loc.toff.data(), c->loc.toff.size() * 8);
    else if (nm == "loc_voff") put(c->loc.voff.data(), c->loc.voff.size() * 8);
    else if (nm == "seg_off") put(c->seg_off.data(), c->seg_off.size() * 8);
    else if (nm == "xv_off") put(c->ls.xv_off.data(), c->ls.xv_off.size() * 8);
    else if (nm == "xv_vert") put(c->ls.xv_vert.data(), c->ls.xv_vert.size() * 4);
    else if (nm == "loc_vlen") {
      const int64_t v = c->loc.vlen;
      put(&v, 8);
    } else if (nm == "mlp_features") {
      auto v = c->d_feat.download(c->stream);
      put(v.data(), v.size() * 4);
    } else if (nm == "eig_V") {
      auto v = c->eigV.download(c->stream);
      put(v.data(), v.size() * 8);
    } else if (nm == "eig_nq") put(c->eig_nq.data(), c->eig_nq.size() * 4);
    else if (nm == "lobpcg_iters") put(c->lobpcg_iters.data(), c->lobpcg_iters.size() * 4);
    else if (nm == "setup_stages") put(c->stage_s, sizeof(c->stage_s));
    else if (nm == "coarse_steps") {
      const std::vector<double> v = geneo::mf_step_profile(c);
      put(v.data(), v.size() * 8);
    }
    else if (nm == "autotune") {
      std::vector<double> v;
      for (const auto &r : c->tune) {
        double row[12];
        for (double &q : row) q = std::nan("");
        row[0] = r.target == "local" ? 0.0 : r.target == "gradient" ? 1.0 : 2.0;
        row[1] = r.precision;
        row[2] = r.chosen;
        row[3] = r.from_cache ? 1.0 : 0.0;
        for (size_t k = 0; k < r.ms.size() && k < 8; ++k) row[4 + k] = r.ms[k];
        v.insert(v.end(), row, row + 12);
      }
      put(v.data(), v.size() * 8);
    }
    else if (nm == "lobpcg_iters_first") put(c->lobpcg_iters0.data(), c->lobpcg_iters0.size() * 4);
    else if (nm == "k0k1") {
      int32_t k[2] = {c->dec.k0, c->dec.k1};
      put(k, 8);
    } else
      return fail(GENEO_ERR_INVALID_ARG, "unknown export name: " + nm);
    if (size) *size = (int64_t)buf.size();
    if (dst) {
      if (cap < (int64_t)buf.size()) return fail(GENEO_ERR_INVALID_ARG, "buffer too small");
      if (!buf.empty()) std::memcpy(dst, buf.data(), buf.size());
    }
    return GENEO_OK;
  });
}

int geneo_mlp_create(uint64_t seed, geneo_mlp **out) {
  if (!out) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  return guarded([&]() {
    auto h = new geneo_mlp();
    try {
      h->m = geneo::mlp_create(seed);
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
    return GENEO_OK;
  });
}

void geneo_mlp_destroy(geneo_mlp *mlp) {
  if (!mlp) return;
  geneo::mlp_destroy(mlp->m);
  delete mlp;
}

int64_t geneo_mlp_param_count(void) { return geneo::mlp_param_count(); }

int geneo_mlp_get_params(const geneo_mlp *mlp, float *host) {
  if (!mlp || !host) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  return guarded([&]() {
    auto w = geneo::mlp_get(mlp->m);
    std::memcpy(host, w.data(), w.size() * sizeof(float));
    return GENEO_OK;
  });
}

int geneo_mlp_set_params(geneo_mlp *mlp, const float *host) {
  if (!mlp || !host) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  return guarded([&]() {
    geneo::mlp_set(mlp->m, std::vector<float>(host, host + geneo::mlp_param_count()));
    return GENEO_OK;
  });
}

int geneo_mlp_loss_grad(geneo_mlp *mlp, geneo_ctx *c, double *loss, float *grad_host, void *s) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!mlp || !c) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  return guarded([&]() {
    const double l = geneo::mlp_loss_grad(mlp->m, c, as_stream(s));
    if (loss) *loss = l;
    if (grad_host) {
      auto g = geneo::mlp_grad_host(mlp->m, as_stream(s));
      std::memcpy(grad_host, g.data(), g.size() * sizeof(float));
    }
    return GENEO_OK;
  });
}

int geneo_mlp_train(geneo_mlp *mlp, geneo_ctx *c, int32_t steps, double lr, double *loss_host,
                    void *s) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!mlp || !c) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  if (steps < 0 || !(lr > 0)) return fail(GENEO_ERR_INVALID_ARG, "steps >= 0, lr > 0");
  return guarded([&]() {
    for (int i = 0; i < steps; ++i) {
      const double l = geneo::mlp_loss_grad(mlp->m, c, as_stream(s));
      if (loss_host) loss_host[i] = l;
      geneo::mlp_adam(mlp->m, lr, as_stream(s));
    }
    GENEO_CUDA(cudaStreamSynchronize(as_stream(s)));
    return GENEO_OK;
  });
}

int geneo_mlp_infer(const geneo_mlp *mlp, geneo_ctx *c, double *X, void *s) {
  if (c && c->host_only) return fail(GENEO_ERR_STATE, "topology-only context");
  if (!mlp || !c || !X) return fail(GENEO_ERR_INVALID_ARG, "null argument");
  return guarded([&]() {
    geneo::mlp_infer(mlp->m, c, X, as_stream(s));
    return GENEO_OK;
  });
}

const char *geneo_last_error(void) { return g_last_error.c_str(); }

const char *geneo_strerror(int s) {
  switch (s) {
    case GENEO_OK: return "ok";
    case GENEO_NOT_CONVERGED: return "not converged";
    case GENEO_ERR_INVALID_ARG: return "invalid argument";
    case GENEO_ERR_CUDA: return "CUDA error";
    case GENEO_ERR_OOM: return "out of memory";
    case GENEO_ERR_NOT_SPD: return "matrix not positive definite";
    case GENEO_ERR_BREAKDOWN: return "Krylov breakdown";
    case GENEO_ERR_TIMEOUT: return "device wait timed out";
    case GENEO_ERR_STATE: return "invalid state";
    default: return "unknown status";
  }
}

}  // extern "C"
