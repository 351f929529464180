// Independent problems composed into one grid (host only).  Problem p is
// placed at x = y = 0 and z offset zoff[p], one inactive cell layer above the
// previous problem; its gamma is folded into eps (the composite has gamma =
// 1) and its cubic cells of side h_p are mapped onto the composite's side H
// (the smallest h_p).  With lowest-order edge elements on a tetrahedron the
// curl-curl term scales as 1/h, the mass term as h and the load as h^2, so
// mu^-1 / r, gamma eps r and f r^2 with r = h_p / H reproduce the problem's
// own matrix and load.  Each problem keeps its own subdomains through the
// composite's explicit cell partition (its boxes, or its own cell_part,
// offset past the previous problems' parts).
#pragma once
#include <cstdint>
#include <vector>

#include "common.cuh"

namespace geneo {

struct Composite {
  int32_t nx = 0, ny = 0, nz = 0;
  double h = 0;
  std::vector<uint8_t> active;
  std::vector<double> mu_inv, eps;
  std::vector<int32_t> part, zoff;
};

// Sizes only (nx, ny, nz, h, zoff) when arrays is false.  Throws Error
// (INVALID_ARG) on inconsistent input.
void compose_problems(int32_t nprob, const geneo_problem *probs, bool arrays, Composite &out);

// f_slot[p]: host [nrhs][nverts_p][7][3] of problem p (NULL: zero load);
// out: host [nrhs][nverts][7][3] of the composite, overwritten.
void compose_field(int32_t nprob, const geneo_problem *probs, const Composite &cmp,
                   const double *const *f_slot, int32_t nrhs, double *out);

}  // namespace geneo
