// Entry points between the C-ABI layer and the set-up / solve modules.
#pragma once
#include "ctx.hpp"

namespace geneo {

void setup_all(geneo_ctx *c);
void assemble_rhs(geneo_ctx *c, const double *fslot_host, double *b, cudaStream_t s);
void check_device_error(geneo_ctx *c, cudaStream_t s);
// GenEO eigenvectors of every subdomain (batched LOBPCG); appends columns
// to the coarse basis
void geneo_eigenvectors(geneo_ctx *c);

void spmv(geneo_ctx *c, const double *x, double *y, cudaStream_t s);
void local_solve(geneo_ctx *c, const double *r, double *w, cudaStream_t s);
void coarse_solve(geneo_ctx *c, const double *r, double *y, cudaStream_t s);
void apply_preconditioner(geneo_ctx *c, const double *r, double *z, cudaStream_t s);
int pcg(geneo_ctx *c, const double *b, double *x, double tol, int maxit, geneo_solve_info *info,
        cudaStream_t s);

}  // namespace geneo
