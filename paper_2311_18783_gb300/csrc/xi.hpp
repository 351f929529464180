// Local operators of every subdomain shared by the GenEO eigensolver and the
// split (mixed-precision) local solves: A_j and A_j^Neu on the local CSR,
// the Boolean partition of unity D_j, the gradient structure G_j of the kept
// vertices, S_j^-1 = (G_j^T A_j G_j)^-1 and S_Bj^-1 = (G_j^T A_j^Neu G_j)^-1
// (tile-packed, one matrix per subdomain) and the element data used to form
// G^T A x and A G w per tetrahedron.
#pragma once
#include "dense.cuh"

namespace geneo {

struct XiOp {
  int64_t vlen = 0, vlenS = 0, nslots = 0, nv = 0;
  DevBuf<int32_t> slot_sub, vslot_sub, pos_sub, ghead, gtail, srow;
  DevBuf<int8_t> ssgn;
  DevBuf<int64_t> Noff, lrp, sptr, xvoff;
  DevBuf<int32_t> lcol;
  DevBuf<double> aval, nval, dmask;
  TileBatch sb;
  DevBuf<double> s_inv;   // S_j^-1,   S_j = G_j^T A_j G_j
  DevBuf<float> s_inv32;  // S_j^-1 rounded to float32 (split local solves, optional)
  DevBuf<double> sn_inv;  // S_Bj^-1,  S_Bj = G_j^T A_j^Neu G_j (same layout)
  // column-tetrahedron lists of the local gradient columns (Dirichlet: all
  // tetrahedra touching N_j; Neumann: those of Omega_j) and per-entry local
  // indices of the tetrahedron's six edges
  DevBuf<int64_t> ctp_d, ctp_n, col_out;
  DevBuf<int32_t> ctt_d, ctt_n, lidx_d, lidx_n, col_sub;
  DevBuf<double> ct_d, ct_n, tcurl, tmass;
  // per local row: tetrahedra containing it (for A_j G w element by element)
  DevBuf<int64_t> rptr;
  DevBuf<int32_t> rtet, rlidx, rvidx;
  DevBuf<int8_t> rpos;
  DevBuf<double> u1, u2, u3;  // vertex vectors of the split local solves
  // gradient shift (A_j replaced by A_j + rho_j A_j G_j S_j^-1 G_j^T A_j before
  // inversion): rho_j, 1 / (1 + rho_j) and rho_j / (1 + rho_j) per subdomain
  bool shifted = false;
  DevBuf<double> rho, gfac, gsc64;
};

}  // namespace geneo
