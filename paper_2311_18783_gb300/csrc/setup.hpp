// Entry points between the C-ABI layer and the set-up / solve modules.
#pragma once
#include "ctx.hpp"

namespace geneo {

// Sparse columns for a Galerkin product X^T A X, each column assigned to a
// matrix of a tile batch and a local index in it.
struct Columns {
  std::vector<int64_t> ptr{0};
  std::vector<int32_t> row;       // unknowns
  std::vector<double> val;
  std::vector<int32_t> mat, loc;  // target matrix and local index
  // true: only tetrahedra of subdomain Omega_mat enter (a Neumann matrix,
  // Sec. 2), else every tetrahedron touching the column
  bool neumann = false;
};

// Galerkin plan: column-tetrahedron entries and the lower pattern of X^T A X
struct GalerkinPlan {
  int64_t ncol = 0;
  std::vector<int64_t> pptr;
  std::vector<int32_t> pcol;
  DevBuf<int64_t> dpp, dctp;
  DevBuf<int32_t> dpc, dctt;
  DevBuf<double> dct;
};
void galerkin_plan(geneo_ctx *c, const Columns &X, GalerkinPlan &P, cudaStream_t s);
// vals[q] for every pattern entry (device array of pcol.size() doubles)
void galerkin_values(GalerkinPlan &P, double *vals, cudaStream_t s);

// X^T A X summed per tetrahedron (curl-curl part through the curl of each
// column on the tetrahedron), written into the tile-packed batch.
void galerkin_tiles(geneo_ctx *c, const Columns &X, TileBatch &b, double *tiles, cudaStream_t s);
// Column-tetrahedron lists and entries (15 doubles: scaled curl of the column
// on the tetrahedron, its six local values, gamma eps M_T times them).
void coltet_build(geneo_ctx *c, const Columns &X, std::vector<int64_t> &ct_ptr,
                  std::vector<int32_t> &ct_tet, DevBuf<int64_t> &dctp, DevBuf<int32_t> &dctt,
                  DevBuf<double> &dct, cudaStream_t s);
// per tetrahedron: sqrt(mu^-1 |T|) curl W_e for the six edges (18 doubles)
// and gamma eps M_T (36 doubles)
void tet_operators(geneo_ctx *c, DevBuf<double> &tcurl, DevBuf<double> &tmass, cudaStream_t s);

void setup_all(geneo_ctx *c);
// times every candidate SYMV configuration on the context's tile batches and
// keeps the fastest (autotune.cu)
void autotune_symv(geneo_ctx *c);
// times the sparse coarse solve as one launch per level and phase and as one
// cooperative launch, keeps the faster (c->mf_persist)
void autotune_coarse(geneo_ctx *c);
void autotune_clear_cache();
// Host part only: topology, decomposition, components, local structure and,
// for a host-only context, the split near-kernel columns.  No CUDA call.
void setup_topology(geneo_ctx *c);
void assemble_rhs(geneo_ctx *c, const double *fslot_host, double *b, cudaStream_t s);
void check_device_error(geneo_ctx *c, cudaStream_t s);
// GenEO eigenvectors of every subdomain (batched LOBPCG); appends columns
// to the coarse basis
void geneo_eigenvectors(geneo_ctx *c);
// builds the local operators of every subdomain (see xi.hpp)
void build_xi_operator(geneo_ctx *c, XiOp &op, cudaStream_t s);
// float32 C_j = (I - xi_j) A_j^-1 of every subdomain (needs the float64 inverse)
void build_split_factors(geneo_ctx *c);
// yl += G_j S_j^-1 G_j^T xl, float64 gradient part of the split local solve
void split_gradient_apply(geneo_ctx *c, const double *xl, double *yl, cudaStream_t s, int k = 1,
                          const double *scale = nullptr);
void apply_gradient_shift(geneo_ctx *c);
// y = A_j^Neu x for k columns of local vectors (the right-hand operator B of
// the local generalised eigenproblems)
void apply_neumann(geneo_ctx *c, const double *x, double *y, int k, cudaStream_t s);

// learned warm start (mlp.cu)
struct Mlp;
int mlp_param_count();
Mlp *mlp_create(uint64_t seed);
void mlp_destroy(Mlp *M);
std::vector<float> mlp_get(const Mlp *M);
void mlp_set(Mlp *M, const std::vector<float> &w);
void mlp_infer(const Mlp *M, geneo_ctx *c, double *X, cudaStream_t s);
double mlp_loss_grad(Mlp *M, geneo_ctx *c, cudaStream_t s);
void mlp_adam(Mlp *M, double lr, cudaStream_t s);
std::vector<float> mlp_grad_host(const Mlp *M, cudaStream_t s);
void build_mlp_features(geneo_ctx *c);
void split_tc_apply(geneo_ctx *c, const double *xl, double *yl, double *xp, cudaStream_t s, int k,
                    cudaEvent_t e0, cudaEvent_t e1);

// multifrontal coarse factor: set-up, solve y = E^-1 t (column order), sizes.
// With `schur`, only the fronts below the root are factored and the root's
// pivot block after the extend-adds, E_hh - E_hg E_gg^-1 E_gh on the GenEO
// columns h (dense, row-major), is returned with the diagonal of E_hh; the
// context keeps no factor.
struct MfSchur {
  int64_t nh = 0;
  std::vector<double> S, diag;
};
void mf_setup(geneo_ctx *c, MfSchur *schur = nullptr);
void mf_solve(geneo_ctx *c, const double *t, double *y, cudaStream_t s, int k = 1);
void mf_reserve(geneo_ctx *c, int k);
int mf_launches_per_solve(const geneo_ctx *c);
bool mf_single_launch_available(const geneo_ctx *c);
// per step of the single-launch coarse solve: kind, level, items, factor bytes,
// SM cycles of CTA 0 in the last profiled solve
std::vector<double> mf_step_profile(const geneo_ctx *c);
int64_t mf_factor_bytes(const geneo_ctx *c);
// algorithmic bytes of one coarse solve: every factor tile the solve reads
int64_t mf_solve_bytes(const geneo_ctx *c);

// Solve path; k right-hand sides stored as k consecutive columns of length n
// (local vectors: columns of loc.vlen).
void reserve_rhs(geneo_ctx *c, int k);
// bfloat16 local factors on the tensor cores (block right-hand sides)
bool tc_supported(const geneo_ctx *c);
void build_bf16_factors(geneo_ctx *c);
int64_t tc_factor_bytes(const geneo_ctx *c);
void tc_symm(geneo_ctx *c, const double *xl, double *yl, int k, cudaStream_t s, cudaEvent_t e0,
             cudaEvent_t e1);
void spmv(geneo_ctx *c, const double *x, double *y, cudaStream_t s, int k = 1);
// y = b - A x (k columns), the same SpMV kernel
void residual(geneo_ctx *c, const double *x, const double *b, double *y, cudaStream_t s,
              int k = 1);
// the SELL-32-256 copy of A used by spmv and residual (from the CSR values)
void build_sell(geneo_ctx *c, cudaStream_t s);
void local_solve(geneo_ctx *c, const double *r, double *w, cudaStream_t s, int k = 1);
// y = Z E^-1 Z^T r (+ add, when given)
void coarse_solve(geneo_ctx *c, const double *r, double *y, cudaStream_t s, int k = 1,
                  const double *add = nullptr);
void apply_preconditioner(geneo_ctx *c, const double *r, double *z, cudaStream_t s, int k = 1);
// one-coarse-solve form for residuals with Z^T r = 0: w + Z E^-1 Z^T (r - A w)
void apply_balanced(geneo_ctx *c, const double *r, double *z, cudaStream_t s, int k = 1);
int pcg(geneo_ctx *c, const double *b, double *x, double tol, int maxit, geneo_solve_info *info,
        cudaStream_t s, int k = 1);
// PCG followed by nref refinement steps with accurate (twice the working
// precision) residuals; info->relres is the accurate relative residual
int pcg_refined(geneo_ctx *c, const double *b, double *x, double tol, int maxit, int nref,
                geneo_solve_info *info, cudaStream_t s);
// right-preconditioned restarted GMRES(restart) with M^-1_AS,2
int gmres(geneo_ctx *c, const double *b, double *x, double tol, int maxit, int restart,
          geneo_solve_info *info, cudaStream_t s);
// one PCG per independent component (contiguous unknown ranges), same launches
int pcg_segments(geneo_ctx *c, const double *b, double *x, double tol, int maxit,
                 geneo_solve_info *info, cudaStream_t s);

}  // namespace geneo
