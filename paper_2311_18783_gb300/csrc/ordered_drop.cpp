// Ordered Cholesky with drops on the host (see ordered_drop.hpp).
//
// Panels of kPanel columns.  For a panel [p0, p1):
//  A. its diagonal block is factored column by column (serial);
//  B. the rows below it get their panel entries L_rk (parallel over rows);
//  C. the trailing block r, c >= p1 is updated with the panel's kept
//     columns in ascending order (parallel over rows).
// An entry (r, c) thus receives -= L_rq L_cq for every kept q < c in
// ascending q, exactly like the column-by-column definition.
#include "ordered_drop.hpp"

#include <algorithm>
#include <cmath>
#include <thread>

namespace geneo {

namespace {

constexpr int64_t kPanel = 64;
constexpr int64_t kChunk = 256;  // trailing columns per L1-resident block

template <class F>
void parallel_rows(int64_t lo, int64_t hi, int nt, F &&f) {
  if (hi <= lo) return;
  if (nt <= 1 || hi - lo < 64) {
    for (int64_t r = lo; r < hi; ++r) f(r);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(nt);
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t]() {
      for (int64_t r = lo + t; r < hi; r += nt) f(r);
    });
  for (auto &x : th) x.join();
}

}  // namespace

std::vector<int64_t> ordered_drop(const std::vector<double> &S, const std::vector<double> &diag,
                                  int64_t nh, double tol, int nthreads,
                                  std::vector<double> *pivots) {
  int nt = nthreads;
  if (nt <= 0) nt = (int)std::min<unsigned>(64, std::max(1u, std::thread::hardware_concurrency()));
  std::vector<double> W(S.begin(), S.begin() + nh * nh);  // becomes L (lower part)
  std::vector<int64_t> keep;
  std::vector<uint8_t> kept(nh, 0);
  if (pivots) pivots->assign(nh, 0.0);
  std::vector<double> Lt;  // panel columns, transposed: Lt[j * nh + c] = L_c,q_j
  for (int64_t p0 = 0; p0 < nh; p0 += kPanel) {
    const int64_t p1 = std::min(nh, p0 + kPanel);
    std::vector<int64_t> pk;  // kept columns of this panel
    // A: diagonal block, column by column
    for (int64_t k = p0; k < p1; ++k) {
      double piv = W[k * nh + k];
      for (int64_t q : pk) piv -= W[k * nh + q] * W[k * nh + q];
      if (pivots) (*pivots)[k] = piv;
      if (!(piv >= tol * diag[k])) continue;
      const double d = std::sqrt(piv);
      W[k * nh + k] = d;
      for (int64_t r = k + 1; r < p1; ++r) {
        double v = W[r * nh + k];
        for (int64_t q : pk) v -= W[r * nh + q] * W[k * nh + q];
        W[r * nh + k] = v / d;
      }
      pk.push_back(k);
      keep.push_back(k);
      kept[k] = 1;
    }
    if (pk.empty() || p1 == nh) continue;
    // B: the panel entries of the rows below the panel
    parallel_rows(p1, nh, nt, [&](int64_t r) {
      double *wr = W.data() + r * nh;
      for (size_t a = 0; a < pk.size(); ++a) {
        const int64_t k = pk[a];
        double v = wr[k];
        for (size_t b = 0; b < a; ++b) v -= wr[pk[b]] * W[k * nh + pk[b]];
        wr[k] = v / W[k * nh + k];
      }
    });
    // C: trailing update with the kept panel columns, ascending
    const int64_t nk = (int64_t)pk.size();
    Lt.assign((size_t)nk * nh, 0.0);
    for (int64_t j = 0; j < nk; ++j)
      for (int64_t c = p1; c < nh; ++c) Lt[j * nh + c] = W[c * nh + pk[j]];
    parallel_rows(p1, nh, nt, [&](int64_t r) {
      double *wr = W.data() + r * nh;
      for (int64_t c0 = p1; c0 <= r; c0 += kChunk) {
        const int64_t c1 = std::min(r + 1, c0 + kChunk);
        for (int64_t j = 0; j < nk; ++j) {
          const double a = wr[pk[j]];
          const double *lt = Lt.data() + j * nh;
          for (int64_t c = c0; c < c1; ++c) wr[c] -= a * lt[c];
        }
      }
    });
  }
  return keep;
}

}  // namespace geneo
