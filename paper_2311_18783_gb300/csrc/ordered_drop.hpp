// Ordered Cholesky with drops (host): the GenEO independence filter.
//
// Z must be a full-rank basis of V_G + V_GenEO (Sec. 3.2, eq. "V0GenEOAS").
// Given the GenEO Schur complement S = E_hh - E_hg E_gg^-1 E_gh (nh x nh,
// row-major, symmetric) and the diagonal of E_hh, the columns are taken in
// order; column k is kept when its pivot in the Cholesky of S restricted to
// the kept columns before it, S_kk - sum_{q kept, q < k} L_kq^2, is at least
// tol * diag[k], and dropped otherwise.
//
// Blocked and multi-threaded, but every entry of L receives the same
// floating-point operations in the same order as the column-by-column
// (left-looking) definition, so the result does not depend on nthreads.
#pragma once
#include <cstdint>
#include <vector>

namespace geneo {

// Returns the kept columns in ascending order; pivots (optional) gets the
// pivot of every column (before the test, so dropped ones are kept too).
// nthreads <= 0 selects the hardware concurrency (at most 64).
std::vector<int64_t> ordered_drop(const std::vector<double> &S, const std::vector<double> &diag,
                                  int64_t nh, double tol, int nthreads = 0,
                                  std::vector<double> *pivots = nullptr);

}  // namespace geneo
