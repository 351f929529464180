/*
 * geneo.h -- C-ABI of the GB300 (sm_103a) library for the two-level
 * GenEO-type additive Schwarz preconditioner of positive Maxwell problems.
 *
 * Method: Bootland, Dolean, Nataf, Tournier, "A robust and adaptive
 * GenEO-type domain decomposition preconditioner for H(curl) problems in
 * three-dimensional general topologies" (arXiv 2311.18783).
 *
 *   problem   curl(mu^-1 curl E) + gamma eps E = f, E x n = 0
 *             (Sec. 1, eq. "positivemaxwell"), discretised with lowest-order
 *             Nedelec edge elements into A U = (K + gamma M) U = f
 *             (Sec. 1, eq. "discretemaxwell"; Sec. 2, eq. "bilinearformposmax");
 *   method    M^-1_AS,2 = Z E^-1 Z^T + (I - P0) sum_i R_i^T A_i^-1 R_i (I - P0^T)
 *             (Sec. 2, eq. "AS2"; closed form at the end of Sec. 3.2), with
 *             Z spanning the split near-kernel space (Sec. 2, definition
 *             "near-kernelCS") plus the GenEO eigenvectors of the filtered
 *             generalised eigenproblem (Sec. 3.2, GEVP "tauthresholdAS",
 *             eq. "eigAtildeBAS") with eigenvalues above the threshold;
 *   Krylov    preconditioned conjugate gradients (A is SPD, Sec. 2, and
 *             M^-1_AS,2 is symmetric, eq. "AS2").
 *
 * Mesh: a structured grid of nx*ny*nz cubic cells, each split into six Kuhn
 * tetrahedra; cells are numbered c = i + nx*(j + ny*k) and vertices
 * v = i + (nx+1)*(j + (ny+1)*k).  Edges run from the lower to the higher
 * vertex id along one of seven positive directions DIRS = {x, y, z, x+y,
 * x+z, y+z, x+y+z} (in that order), so an edge is identified by its slot
 * (v, d).  Unknowns are the edges that do not lie on the boundary (Dirichlet
 * E x n = 0, eliminated), numbered in lexicographic (tail, head) order.
 *
 * Conventions of every entry point:
 *  - "host" pointers are caller-owned CPU memory, only read (or written)
 *    during the call; "device" pointers are caller-owned CUDA global memory
 *    on the context's device, of float64 unless stated otherwise;
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream); work is enqueued on it and the call returns without waiting,
 *    except where a host result is produced (noted per call);
 *  - the return value is GENEO_OK (0) on success, a positive warning, or a
 *    negative error code; geneo_last_error() gives a message.  No exception
 *    or abort crosses this interface.
 *  - all memory the context needs is allocated in geneo_setup and released
 *    by geneo_destroy.  A context is not thread safe; calls that use the
 *    same context must not overlap.
 */
#ifndef GENEO_H
#define GENEO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GENEO_OK 0
#define GENEO_NOT_CONVERGED 1      /* warning: maxit reached, x holds the last iterate */
#define GENEO_ERR_INVALID_ARG (-1)
#define GENEO_ERR_CUDA (-2)
#define GENEO_ERR_OOM (-3)
#define GENEO_ERR_NOT_SPD (-4)     /* a pivot of a factorisation was not positive */
#define GENEO_ERR_BREAKDOWN (-5)   /* PCG: p^T A p <= 0 or not finite */
#define GENEO_ERR_TIMEOUT (-6)     /* a bounded device wait gave up */
#define GENEO_ERR_STATE (-7)       /* call not valid in the context's state */

#define GENEO_PREC_FP64 0          /* local factors stored and applied in float64 */
#define GENEO_PREC_FP32 1          /* split factors (Sec. 2, eq. "inverseBw"): A_j^-1 =
                                      G S^-1 G^T (float64) + (I - xi) A_j^-1 (float32) */
#define GENEO_PREC_BF16 2          /* the same split with (I - xi) A_j^-1 in bfloat16, applied on
                                      the tensor cores with float32 accumulation to blocks of up
                                      to 16 right-hand sides (x rounded to bfloat16); needs
                                      n_j <= 2048 in every subdomain (else INVALID_ARG) */

#define GENEO_COARSE_NONE 0        /* one-level additive Schwarz (eq. "AS") */
#define GENEO_COARSE_SNK 1         /* split near-kernel space (definition "near-kernelCS") */
#define GENEO_COARSE_NK 2          /* global near-kernel G: one gradient column per interior
                                      vertex (Sec. 4, variants AS-NK and AS-NK-GenEO) */

#define GENEO_PENCIL_FILTERED 0    /* GEVP "tauthresholdAS", eq. "eigAtildeBAS" (Sec. 3.2):
                                      (I - xi_0j)^T D_j A_j D_j (I - xi_0j) V = lambda A_j^Neu V,
                                      coarse vectors R_j^T D_j (I - xi_0j) V */
#define GENEO_PENCIL_CLASSICAL 1   /* the classical GenEO pencil of the remark in Sec. 3.2,
                                      eq. "eigGenEOClassis": D_j A_j D_j V = lambda A_j^Neu V,
                                      coarse vectors R_j^T D_j V; for comparison: it has many
                                      gradient-driven eigenvalues above the threshold, most of
                                      them dependent on the split near-kernel columns; its
                                      LOBPCG search directions use the inverse of
                                      A_j^Neu + 1e-10 diag(A_j^Neu) */

#define GENEO_TAU_RECIPROCAL 0     /* select lambda > 1/tau */
#define GENEO_TAU_PAPER 1          /* select lambda > tau (GEVP "tauthresholdAS" literally) */

/* Opaque context: owns every device allocation of one set-up problem. */
typedef struct geneo_ctx geneo_ctx;
typedef struct geneo_mlp geneo_mlp;  /* warm-start network (see the end of this header) */

/* Problem description; arrays are host memory, copied during geneo_setup. */
typedef struct {
  int32_t nx, ny, nz;        /* cells per axis, each >= 1 */
  double hx, hy, hz;         /* cell edge lengths, > 0 */
  const uint8_t *active;     /* [nx*ny*nz] 1 = cell present, 0 = hole */
  const double *mu_inv;      /* [nx*ny*nz] mu^-1 per cell, > 0 */
  const double *eps;         /* [nx*ny*nz] eps per cell, > 0 */
  double gamma;              /* > 0 */
  int32_t px, py, pz;        /* boxes per axis; cell (i,j,k) is in box (i*px/nx, j*py/ny, k*pz/nz) */
  int32_t overlap;           /* layers of cells added around each box (vertex neighbours), >= 1 */
  double tau;                /* GenEO threshold, > 0, read with options.tau_convention */
  const int32_t *cell_part;  /* NULL: the boxes above; else [nx*ny*nz] subdomain id >= 0 of
                                every active cell (px, py, pz ignored).  Independent problems
                                placed in one grid, separated by inactive cells and stacked
                                along z, are solved together by geneo_solve_segments. */
  const uint8_t *natural_faces; /* NULL: E x n = 0 on every boundary face; else [nx*ny*nz]
                                per cell, bit 2a + s (a = 0, 1, 2 for x, y, z; s = 0 lower,
                                1 upper side) marks that face of the cell as a natural
                                (Neumann) boundary when it lies on the boundary (hole
                                surfaces, lateral faces: Sec. 4, mixed boundary conditions);
                                its edges and vertices are then unknowns. */
} geneo_problem;

typedef struct {
  int32_t precision;         /* GENEO_PREC_* */
  int32_t coarse;            /* GENEO_COARSE_* */
  int32_t geneo;             /* 1: add GenEO eigenvectors to the coarse space */
  int32_t tau_convention;    /* GENEO_TAU_* */
  int32_t lobpcg_block;      /* block size of the batched LOBPCG, 1..16 */
  int32_t lobpcg_maxit;      /* iterations per block before giving up */
  double lobpcg_tol;         /* relative eigen-residual tolerance */
  uint64_t seed;             /* initial LOBPCG blocks (counter-based hash) */
  int32_t coarse_dense;      /* 0: sparse multifrontal Cholesky of E (nested dissection);
                                1: explicit dense E^-1 (small coarse spaces, testing) */
  int32_t coarse_leaf;       /* sparse factor: nested-dissection regions of at most this
                                many columns become leaf fronts; 0 selects 256 */
  int32_t use_graph;         /* 1: every PCG iteration after the first replays one CUDA
                                graph captured at the first solve; 0: plain launches */
  int32_t gradient_shift;    /* 1: invert A~_j = A_j + rho_j A_j G_j S_j^-1 G_j^T A_j instead of
                                A_j (same C_j and A_j^-1 exactly, see Sec. 2 eq. "inverseBw";
                                needed when gamma makes A_j numerically singular); 0: off */
  int32_t keep_eigvecs;      /* 1: keep the first 8 locked eigenvectors of every subdomain and
                                the edge features (training data of the warm-start network) */
  const struct geneo_mlp *warm_start;  /* non-NULL: the first LOBPCG block of every subdomain
                                is this network's output on the edge features (needs
                                lobpcg_block == 8); NULL: seeded random block */
  int32_t lobpcg_neumann;    /* 1: LOBPCG for small boxes with high contrast and tiny gamma:
                                the search directions use the explicit inverse of
                                A_j^Neu + 1e-10 diag(A_j^Neu) (the right-hand operator of the
                                GEVP) instead of A_j^-1, the Rayleigh-Ritz step works in the
                                B-Gram basis of [X W P], and a Ritz value that has stayed
                                within 1e-4 relative for five iterations, at least 1% away
                                from tau, counts as converged (float64 residuals of such
                                pencils stall far above lobpcg_tol).  Use with
                                lobpcg_block = 16.  0: off */
  int32_t balanced;          /* 1: PCG in the balanced form: start from x0 = Z E^-1 Z^T b, so
                                Z^T r_k = 0 in exact arithmetic, where the closed form of
                                M^-1_AS,2 (end of Sec. 3.2) reduces to (I - P0) sum_i R_i^T
                                A_i^-1 R_i; applied as w + Z E^-1 Z^T (r - A w), one coarse
                                solve per iteration instead of two (the Z E^-1 Z^T r part,
                                zero in exact arithmetic, corrects the rounding drift of
                                Z^T r_k).  0: x0 = 0 and the literal four-step apply.
                                Switchable later with geneo_use_balanced. */
  int32_t geneo_pencil;      /* GENEO_PENCIL_FILTERED (default) or GENEO_PENCIL_CLASSICAL */
  int32_t autotune;          /* 1: before the eigensolves, time every candidate launch
                                configuration of the streaming SYMV (bulk-copy stages,
                                tiles per barrier pair, warps per CTA, CTAs per SM) on the
                                context's local factors (each stored precision) and S_j^-1
                                blocks, and keep the fastest; after the coarse factor, time
                                both shapes of the sparse coarse solve (one launch per
                                level and phase, one cooperative launch) and keep the
                                faster.  Results are cached per process by target,
                                precision, nrhs and size buckets (geneo_export
                                ("autotune")).  0: the default configurations */
  const char *autotune_cache; /* NULL, or a text file read before tuning and appended with
                                every new result ("key index milliseconds" per line); the
                                string is only read during geneo_setup */
} geneo_options;

typedef struct {
  int64_t nverts, ncells, ntets, nedges;
  int64_t n;                 /* unknowns (interior edges) */
  int64_t nnz;               /* nonzeros of A (CSR, both triangles) */
  int32_t nsub;              /* subdomains */
  int32_t k0, k1;            /* Sec. 2, eq. "k0", and the maximal cell multiplicity */
  int64_t sum_ni;            /* sum of n_i */
  int64_t max_ni;
  int64_t n0;                /* coarse dimension */
  int64_t n0_snk;            /* split near-kernel columns */
  int64_t n0_geneo;          /* GenEO columns kept */
  int64_t local_factor_bytes;  /* bytes of the stored local factors */
  int64_t coarse_factor_bytes; /* bytes of the stored coarse factor */
  double setup_seconds;      /* wall time of geneo_setup */
} geneo_sizes;

typedef struct {
  int32_t iters;
  double relres;             /* ||b - A x|| / ||b|| of the PCG recurrence at exit */
  double seconds;            /* wall time of the solve, including the final synchronisation */
} geneo_solve_info;

/* Fills `opt` with the defaults: FP64, SNK coarse space, GenEO on,
 * reciprocal tau, LOBPCG block 8, 200 iterations, tolerance 1e-8 (a block
 * whose relative residual has stopped decreasing for 10 iterations is
 * accepted below 1e-4: under a 1e6 contrast of mu^-1 the local residuals
 * stall near 1e-6, where the eigenvalues are already accurate to ~1e-10),
 * seed 1,
 * sparse coarse factor, PCG iteration as a CUDA graph. */
void geneo_default_options(geneo_options *opt);

/* Builds topology, decomposition, A, the local factors, the GenEO
 * eigenvectors and the coarse factor on the current CUDA device (Sec. 2-3).
 * Blocks until the set-up has finished.  On success *out owns all device
 * memory of the problem.  Errors: INVALID_ARG (bad sizes, gamma <= 0,
 * overlap < 1, empty mesh), OOM, CUDA, NOT_SPD. */
int geneo_setup(const geneo_problem *prob, const geneo_options *opt, geneo_ctx **out);

/* The host part of geneo_setup only, without any CUDA call (callable without
 * a GPU): mesh, Dirichlet elimination and unknown numbering (Sec. 4 mesh,
 * Sec. 1 eq. "positivemaxwell"), CSR pattern, subdomains with overlap and
 * partition of unity (Sec. 2, eq. "PoU"), k0/k1, independent components and
 * the split near-kernel columns (Sec. 2, definition "near-kernelCS") when
 * opt->coarse is SNK.  The context answers geneo_query and the integer
 * names of geneo_export; every call that needs device data returns STATE.
 * Same arguments and errors as geneo_setup. */
int geneo_setup_topology(const geneo_problem *prob, const geneo_options *opt, geneo_ctx **out);

/* Releases every resource of the context (NULL is allowed). */
void geneo_destroy(geneo_ctx *ctx);

/* Host copy of the sizes. */
int geneo_query(const geneo_ctx *ctx, geneo_sizes *out);

/* b_dev[n] = load l(v) = int f . W_e (Sec. 2) of the source field given per
 * edge slot: f_slot_host is [nverts][7][3] float64 host memory (slots that
 * are not edges are ignored).  f is read as the Whitney interpolant with
 * dofs f_e . (x_head - x_tail), so b = M_1 c (exact for constant f). */
int geneo_assemble_rhs(geneo_ctx *ctx, const double *f_slot_host, double *b_dev, void *stream);

/* y_dev[n] = A x_dev (Sec. 1, eq. "discretemaxwell"), CSR SpMV. */
int geneo_spmv(geneo_ctx *ctx, const double *x_dev, double *y_dev, void *stream);

/* w_dev[n] = sum_i R_i^T A_i^-1 R_i r_dev (Sec. 2, eq. "AS"). */
int geneo_local_solve(geneo_ctx *ctx, const double *r_dev, double *w_dev, void *stream);

/* y_dev[n] = Z E^-1 Z^T r_dev, E = Z^T A Z (Sec. 2); zero if there is no coarse space. */
int geneo_coarse_solve(geneo_ctx *ctx, const double *r_dev, double *y_dev, void *stream);

/* z_dev[n] = M^-1_AS,2 r_dev (Sec. 2, eq. "AS2"; closed form at the end of Sec. 3.2). */
int geneo_apply_preconditioner(geneo_ctx *ctx, const double *r_dev, double *z_dev, void *stream);

/* PCG on A x = b from x = 0 until ||r||/||b|| <= tol or maxit iterations;
 * b_dev, x_dev device [n].  Synchronises `stream` once per iteration to test
 * convergence; `info` (host, may be NULL) receives the iteration count,
 * final relative residual and wall time.  Returns OK, NOT_CONVERGED or
 * BREAKDOWN. */
int geneo_solve(geneo_ctx *ctx, const double *b_dev, double *x_dev, double tol, int32_t maxit,
                geneo_solve_info *info, void *stream);

/* geneo_solve followed by nref (0..16) steps of iterative refinement: each
 * step evaluates r = b - A x as accurately as in twice the working precision
 * (error-free products and sums, the Dot2 algorithm of Ogita, Rump and
 * Oishi), solves A d = r with the same PCG and tolerance, and adds d to x.
 * In float64, b - A x cannot be evaluated below u ||A|| ||x||, and when gamma
 * is small the gradient part of x (of size 1/gamma, Sec. 1) makes that the
 * floor of the forward error of every float64 solve; refinement removes it.
 * b_dev and x_dev must not alias.  info->iters is the PCG iteration count of
 * all solves, info->relres the accurate ||b - A x|| / ||b|| of the returned
 * x (bounded below by the rounding of x itself to float64).  Returns OK,
 * NOT_CONVERGED (some solve reached maxit) or BREAKDOWN. */
int geneo_solve_refined(geneo_ctx *ctx, const double *b_dev, double *x_dev, double tol,
                        int32_t maxit, int32_t nref, geneo_solve_info *info, void *stream);

/* Right-preconditioned restarted GMRES(restart) on A x = b from x = 0 with
 * M^-1_AS,2, the Krylov method of the paper's experiments (Sec. 4: right
 * preconditioning minimises ||b - A x|| itself, whatever the preconditioner);
 * stops when ||b - A x|| <= tol ||b|| (the Arnoldi estimate, confirmed on the
 * true residual at the end of a cycle) or after maxit iterations in all.
 * Keeps 2 restart + 1 vectors of n doubles in the context (allocated at the
 * first call with a larger restart).  b_dev, x_dev device [n], not aliased;
 * info->iters counts Arnoldi steps, info->relres is the true relative
 * residual.  Synchronises `stream` once per iteration.  Returns OK,
 * NOT_CONVERGED or BREAKDOWN. */
int geneo_solve_gmres(geneo_ctx *ctx, const double *b_dev, double *x_dev, double tol,
                      int32_t maxit, int32_t restart, geneo_solve_info *info, void *stream);

/* Launch configurations of the streaming SYMV of the local factors
 * (options.autotune chooses among them): geneo_symv_config_count gives their
 * number for a storage precision (GENEO_PREC_FP32 or GENEO_PREC_FP64; else
 * INVALID_ARG), geneo_use_symv_config selects entry `index` (0 = default)
 * for the context's local factors in that precision.  Every configuration
 * computes the same product; only the association of the column partial
 * sums differs. */
int geneo_symv_config_count(int32_t precision);
int geneo_use_symv_config(geneo_ctx *ctx, int32_t precision, int32_t index);

/* Storage precision of S_j^-1 in the gradient part G_j S_j^-1 G_j^T of the
 * split local inverse (Sec. 2, eq. "inverseBw"), used by the FP32 split
 * solves: GENEO_PREC_FP64 (default) or GENEO_PREC_FP32 (S_j^-1 rounded to
 * float32, float32 accumulation).  S_j^-1 is SPD and its rounding stays in
 * range(G_j), so the split inverse stays SPD: on ker G_j^T it equals C_j,
 * elsewhere the gradient part adds a PSD term.  STATE unless the split
 * factors were built (options.precision FP32 or BF16).  The float64 shifted
 * inverse (options.gradient_shift) always applies its gradient term in
 * float64. */
int geneo_use_gradient_precision(geneo_ctx *ctx, int32_t precision);

/* on = 1 / 0: later PCG solves of the context use the balanced form / the
 * literal form (see geneo_options.balanced).  geneo_apply_preconditioner
 * always applies the literal M^-1_AS,2. */
int geneo_use_balanced(geneo_ctx *ctx, int32_t on);

/* Kernel shape of the sparse coarse solve y = E^-1 t (Sec. 2, E = Z^T A Z;
 * multifrontal factor of the nested-dissection ordering).  on = 1:
 * the whole solve is one cooperative launch whose resident CTAs run the
 * level-by-level steps separated by a bounded grid-wide barrier (a barrier
 * that waits more than about two seconds makes the call return
 * GENEO_ERR_TIMEOUT).  on = 0 (default): one launch per level and phase.
 * Both compute the same operations in the same order and give identical
 * results; options.autotune times both on the context's factor and keeps the
 * faster.  Where the device offers no cooperative launch, on = 1 behaves as
 * on = 0.  INVALID_ARG unless on is 0 or 1. */
int geneo_use_persistent_coarse(geneo_ctx *ctx, int32_t on);

/* Same solve with host buffers: copies b_host[n] to the device, solves, and
 * copies x back to x_host[n] before returning. */
int geneo_solve_host(geneo_ctx *ctx, const double *b_host, double *x_host, double tol,
                     int32_t maxit, geneo_solve_info *info, void *stream);

/* Block right-hand sides: nrhs (1..16) columns stored one after another,
 * R_dev/Z_dev device [nrhs][n].  Z = M^-1_AS,2 R column by column; every
 * stage runs once for all columns (local factors and coarse factor tiles are
 * read once per column block where the kernel allows).  Column j equals the
 * single-column result bit for bit. */
int geneo_apply_preconditioner_block(geneo_ctx *ctx, const double *R_dev, double *Z_dev,
                                     int32_t nrhs, void *stream);

/* nrhs independent PCG solves (Sec. 2: A SPD, M^-1_AS,2 symmetric) sharing
 * the operator, B_dev/X_dev device [nrhs][n].  Each column stops at its own
 * ||r_j|| <= tol ||b_j|| and is frozen while the others continue; column j
 * equals geneo_solve on b_j bit for bit.  info (host, may be NULL) holds nrhs
 * entries.  Returns OK if every column converged, else NOT_CONVERGED or
 * BREAKDOWN (the worst). */
int geneo_solve_block(geneo_ctx *ctx, const double *B_dev, double *X_dev, int32_t nrhs,
                      double tol, int32_t maxit, geneo_solve_info *info, void *stream);

/* Independent problems in one context: the connected components of the
 * active cells (vertex neighbours) are independent systems (A, Z and M^-1_AS,2
 * are block diagonal over them).  When their unknowns are contiguous (the
 * problems are stacked along z), this runs one PCG per component in the same
 * launches: per-component scalars, each component stopping at its own
 * ||r_c|| <= tol ||b_c||.  b_dev, x_dev device [n]; info (host, may be NULL)
 * holds one entry per component (geneo_export("seg_off") gives their unknown
 * ranges).  Returns OK, NOT_CONVERGED or BREAKDOWN (the worst); STATE if the
 * components are not contiguous. */
int geneo_solve_segments(geneo_ctx *ctx, const double *b_dev, double *x_dev, double tol,
                         int32_t maxit, geneo_solve_info *info, void *stream);

/* Composition of independent problems into one grid, host only (no device
 * work; callable without a GPU).  Problem p is placed at x = y = 0 and at
 * z offset zoff[p], one inactive cell layer above problem p-1; the composite
 * grid is max nx x max ny x (sum (nz_p + 1) - 1) cubic cells of side
 * H = min h_p.  Each problem keeps its subdomains through the composite's
 * cell partition (its boxes, or its own cell_part, offset past the parts of
 * the problems before it).  Its gamma is folded into eps (the composite has
 * gamma = 1) and a cell side h_p != H is mapped exactly: lowest-order edge
 * elements give a curl-curl term that scales as 1/h, a mass term as h and a
 * load as h^2 (Sec. 2, eq. "bilinearformposmax"), so mu^-1 / r,
 * gamma eps r and f r^2 with r = h_p / H give the problem's own A and b.
 * A (and Z, M^-1_AS,2) of the composite are block diagonal over the problems.
 * Every problem needs cubic cells and the same overlap and tau.
 *
 * geneo_compose_size: dims = {nx, ny, nz} of the composite, *h = H.
 * geneo_compose: fills host arrays of nx*ny*nz entries (active, mu_inv, eps,
 *   cell_part; cells outside every problem are inactive with mu^-1 = eps = 1)
 *   and, if zoff is not NULL, zoff[nprob].
 * geneo_compose_field: f_slot[p] host [nrhs][nverts_p][7][3] (the edge-slot
 *   load of geneo_assemble_rhs; NULL = zero) into f_out host
 *   [nrhs][nverts][7][3] of the composite (overwritten), scaled by r^2.
 * geneo_setup_batch: geneo_setup of the composite (gamma = 1, overlap and
 *   tau of the problems, the composed cell partition); solve it with
 *   geneo_solve_segments, one PCG per problem, in problem order (a problem
 *   without interior edges has no unknown and no component).
 * Errors: INVALID_ARG (no problem, non-cubic cells, mixed overlap or tau,
 * null arrays, composite above 2^28 cells), and those of geneo_setup. */
int geneo_compose_size(int32_t nprob, const geneo_problem *probs, int32_t *dims, double *h);
int geneo_compose(int32_t nprob, const geneo_problem *probs, uint8_t *active, double *mu_inv,
                  double *eps, int32_t *cell_part, int32_t *zoff);
int geneo_compose_field(int32_t nprob, const geneo_problem *probs, const double *const *f_slot,
                        int32_t nrhs, double *f_out);
int geneo_setup_batch(int32_t nprob, const geneo_problem *probs, const geneo_options *opt,
                      geneo_ctx **out);

/* Selects the local factors used by later solves when the context holds
 * several: GENEO_PREC_FP64 (explicit float64 inverses), GENEO_PREC_BF16 (built
 * when options.precision was BF16, together with the float32 split) or GENEO_PREC_FP32 (the
 * split C_j + G_j S_j^-1 G_j^T, built when options.precision was FP32; the
 * float64 inverses are kept as well).  Returns STATE if they were not built. */
int geneo_use_precision(geneo_ctx *ctx, int32_t precision);

/* Per-stage counters of the solve path, collected while profiling is on. */
typedef struct {
  int64_t launches;          /* kernels this library launched since the last read */
  int64_t local_symv_launches;  /* launches of the local-factor SYMV kernel */
  double local_symv_ms;      /* their summed duration (CUDA events on the caller's stream) */
  int64_t coarse_symv_launches;
  double coarse_symv_ms;
  int64_t local_symv_bytes;  /* algorithmic bytes of one local SYMV launch (stored tiles) */
  int64_t local_symv_flops;  /* algorithmic flops of one local SYMV launch: 2 sum_i n_i^2 */
  int64_t coarse_solve_bytes; /* algorithmic bytes of one sparse coarse solve: the factor
                                tiles (64 x 64 float64) its forward and backward passes read */
} geneo_profile;

/* on != 0: record CUDA events around every SYMV launch (adds two event
 * records per launch) and count launches.  Off by default. */
int geneo_profile_enable(geneo_ctx *ctx, int32_t on);

/* Waits for the recorded events, fills *out with the counters accumulated
 * since the previous read and resets them. */
int geneo_profile_read(geneo_ctx *ctx, geneo_profile *out);

/* Copies the internal array `name` into host memory dst (capacity bytes);
 * *size receives the byte size (call with dst = NULL to query).  For parity
 * tests of the integer and floating-point set-up data.  Names:
 *  "edges"       int32 [nedges][2]  tail, head vertex ids
 *  "dir_edge"    uint8 [nedges]     1 = Dirichlet edge
 *  "dof_edge"    int32 [n]          edge id of each unknown
 *  "dof_vert"    int32 [nvdofs]     interior vertices
 *  "A_rowptr"    int32 [n+1], "A_col" int32 [nnz], "A_val" float64 [nnz]
 *  "N_off"       int64 [nsub+1], "N_idx" int32 [sum n_i]  R_i index sets
 *  "owner"       int32 [n]          subdomain owning each unknown (partition of unity)
 *  "snk_sub", "snk_vert"  int32 [n0_snk]  subdomain and vertex of each SNK column
 *  "geneo_sub"   int32 [n0_geneo], "geneo_lambda" float64 [n0_geneo]
 *  "geneo_found" int32 [nsub]       eigenvalues above the threshold found per subdomain
 *  "Zcol_ptr" int64 [n0+1], "Zcol_row" int32 [nnzZ], "Zcol_val" float64 [nnzZ]
 *  "k0k1"        int32 [2]
 *  "xv_off"      int64 [nsub+1], "xv_vert" int32  kept vertices of G_j per subdomain
 *  "seg_off"     int64 [ncomp+1]    unknown ranges of the independent components
 *  "loc_nt" int32 [nsub], "loc_toff" int64 [nsub+1], "loc_voff" int64 [nsub+1],
 *  "loc_vlen" int64 [1], "loc_f32" float32  tile layout and float32 local factors
 *  "lobpcg_iters", "lobpcg_iters_first" int32 [nsub]  LOBPCG iterations (all, first block)
 *  "setup_stages" float64 [8]       wall seconds of the set-up stages: assembly (with the
 *                                   topology), local inverses, split / bfloat16 factors,
 *                                   GenEO eigensolves, GenEO independence filter, coarse
 *                                   factor, autotuning, total
 *  "autotune"    float64 [targets][12]  per tuned target: target (0 local-factor SYMV,
 *                                   1 S_j^-1 SYMV, 2 coarse solve shape with candidates
 *                                   0 per level and phase, 1 one cooperative launch),
 *                                   precision, chosen candidate, 1 if it came from the
 *                                   cache, then milliseconds per candidate (NaN past the
 *                                   last)
 *  "coarse_steps" float64 [steps][5]  per step of the single-launch coarse solve
 *                                   (geneo_use_persistent_coarse): kind (0 permutation in,
 *                                   1 gather, 2..5 tile phase 0..3, 6 permutation out),
 *                                   tree level (-1 for the permutations), items, factor
 *                                   bytes read, SM cycles of the first CTA from the step's
 *                                   start to the next one's in the last such solve run
 *                                   with profiling on (zeros before one); empty without
 *                                   a sparse coarse factor
 *  "mlp_features" float32 [loc_vlen][5], "eig_V" float64 [8][loc_vlen],
 *  "eig_nq" int32 [nsub]            warm-start features and training targets
 * Returns INVALID_ARG for an unknown name or a too small buffer, STATE for a
 * device-backed name on a topology-only context. */
int geneo_export(const geneo_ctx *ctx, const char *name, void *dst, int64_t capacity,
                 int64_t *size);

/* Allocation-free symmetric matrix-vector product, for callers that cannot
 * allocate device memory at the point of the call (code inside a memory pool
 * or arena that forbids new allocations, real-time loops where cudaMalloc or
 * cudaFree would synchronise or stall, hosts whose allocator owns all device
 * memory).  The paper has no counterpart: this is a service entry point.
 *
 * y_dev[dim] = T x_dev for one symmetric matrix T given in the tile-packed
 * layout used for the local factors: nt = ceil(dim/64) tiles per side, tile
 * (I, J), J <= I, a full 64x64 row-major block at element offset
 * (I(I+1)/2 + J) * 4096 of tiles_dev (float64, device, 16-byte aligned;
 * x_dev and y_dev 8-byte aligned);
 * diagonal tiles hold both triangles; entries past dim must be finite
 * (zero).  1 <= dim <= 4096.
 *
 * No allocation: the only scratch (partial sums and an error word, 1.07 MB)
 * is a fixed array that every GPU loading the library keeps until exit.
 * The first call on a device looks up that array's device address and sets
 * the kernel's shared-memory limit, so it must come before any stream
 * capture.  All calls share the array and later calls overwrite it: calls
 * that overlap on the GPU (other threads, other streams) race.  The call
 * waits for `stream` before returning.  Errors: INVALID_ARG (null or
 * misaligned pointer, dim outside [1, 4096]), TIMEOUT (a bounded device wait
 * gave up and the copies in flight were drained), CUDA (a CUDA call failed,
 * or a drain wait gave up as well: a copy may still have been writing shared
 * memory when the kernel exited, so treat the CUDA context as lost). */
int geneo_symv_packed_noalloc(const double *tiles_dev, int32_t dim, const double *x_dev,
                              double *y_dev, void *stream);

/* ---- Learned warm start of the local eigensolves (the GEVPs of Sec. 3.2,
 * GEVP "tauthresholdAS").  The paper solves them directly; this network
 * (5 -> 128 -> 128 -> 8, ReLU, bfloat16 weights, float32 accumulation) maps
 * per-edge features (log10 mu^-1 of the edge's tetrahedra / 6, hop distance
 * to the subdomain's artificial boundary / 8, |unit edge direction|) to the
 * first LOBPCG block.  It is trained on eigenvectors the exact set-up
 * produced (options.keep_eigvecs = 1) with the subspace loss
 *   L_j = ||(I - V V^T B) X||^2 / ||X||^2 + 0.1 ||X^T B X - I||^2
 * averaged over subdomains with eigenvectors (B = A_j^Neu, V the locked
 * eigenvectors, X the network's block).  The network lives on the device that
 * was current at creation. */
int geneo_mlp_create(uint64_t seed, geneo_mlp **out);  /* He-normal weights, zero biases */
void geneo_mlp_destroy(geneo_mlp *mlp);
int64_t geneo_mlp_param_count(void);                   /* 18312 */
/* float32 master parameters, layout W1[128][5] b1[128] W2[128][128] b2[128]
 * W3[8][128] b3[8]; host arrays of geneo_mlp_param_count() floats */
int geneo_mlp_get_params(const geneo_mlp *mlp, float *host);
int geneo_mlp_set_params(geneo_mlp *mlp, const float *host);  /* also resets Adam */
/* loss on ctx's kept eigenvectors and its parameter gradient (host, may be
 * NULL), with the network's current bfloat16 weights */
int geneo_mlp_loss_grad(geneo_mlp *mlp, geneo_ctx *ctx, double *loss, float *grad_host,
                        void *stream);
/* `steps` full-batch Adam steps (learning rate lr) on ctx's kept
 * eigenvectors; loss_host[steps] (may be NULL) receives the loss before each */
int geneo_mlp_train(geneo_mlp *mlp, geneo_ctx *ctx, int32_t steps, double lr, double *loss_host,
                    void *stream);
/* X_dev (device, 8 x loc_vlen doubles, loc_vlen from geneo_export("loc_vlen"))
 * = the network's block on ctx's padded local rows (needs ctx features) */
int geneo_mlp_infer(const geneo_mlp *mlp, geneo_ctx *ctx, double *X_dev, void *stream);

/* Message of the last error of this thread. */
const char *geneo_last_error(void);

/* Static text of a status code. */
const char *geneo_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* GENEO_H */
