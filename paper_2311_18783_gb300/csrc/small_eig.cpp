// Small dense symmetric eigenproblems of the batched LOBPCG, on the host
// (see small_eig.hpp).  Plain C++, no CUDA.
#include "small_eig.hpp"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>

namespace geneo {

// Cyclic Jacobi rotations until the off-diagonal mass is below 1e-32 of the
// total (at most 60 sweeps).
void host_sym_eig(int n, std::vector<double> &a, std::vector<double> &w,
                  std::vector<double> &v) {
  v.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      const double h = 0.5 * (a[(size_t)i * n + j] + a[(size_t)j * n + i]);
      a[(size_t)i * n + j] = a[(size_t)j * n + i] = h;
    }
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0, tot = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double x = a[(size_t)i * n + j] * a[(size_t)i * n + j];
        tot += x;
        if (i != j) off += x;
      }
    if (!(off > 1e-32 * tot)) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
        const double z = (aqq - app) / (2.0 * apq);
        const double t = (z >= 0 ? 1.0 : -1.0) / (std::fabs(z) + std::sqrt(1.0 + z * z));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
        for (int r = 0; r < n; ++r) {
          const double arp = a[(size_t)r * n + p], arq = a[(size_t)r * n + q];
          a[(size_t)r * n + p] = cs * arp - sn * arq;
          a[(size_t)r * n + q] = sn * arp + cs * arq;
        }
        for (int r = 0; r < n; ++r) {
          const double apr = a[(size_t)p * n + r], aqr = a[(size_t)q * n + r];
          a[(size_t)p * n + r] = cs * apr - sn * aqr;
          a[(size_t)q * n + r] = sn * apr + cs * aqr;
        }
        for (int r = 0; r < n; ++r) {
          const double vrp = v[(size_t)r * n + p], vrq = v[(size_t)r * n + q];
          v[(size_t)r * n + p] = cs * vrp - sn * vrq;
          v[(size_t)r * n + q] = sn * vrp + cs * vrq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = a[(size_t)i * n + i];
}

void general_rr(int ns, int ld, int kout, const double *H, const double *M, double *theta,
                double *C) {
  std::vector<double> a((size_t)ns * ns), e, U;
  for (int i = 0; i < ns; ++i)
    for (int j = 0; j < ns; ++j) a[(size_t)i * ns + j] = M[(size_t)i * ld + j];
  host_sym_eig(ns, a, e, U);
  double emax = 0;
  for (double x : e) emax = std::max(emax, x);
  std::vector<int> keep;
  for (int i = 0; i < ns; ++i)
    if (e[i] > 1e-12 * emax) keep.push_back(i);
  const int r = (int)keep.size();
  std::vector<double> F((size_t)ns * std::max(r, 1), 0.0);
  for (int i = 0; i < ns; ++i)
    for (int c = 0; c < r; ++c)
      F[(size_t)i * r + c] = U[(size_t)i * ns + keep[c]] / std::sqrt(e[keep[c]]);
  // Hr = F^T H F
  std::vector<double> HF((size_t)ns * std::max(r, 1), 0.0), Hr((size_t)r * r, 0.0);
  for (int i = 0; i < ns; ++i)
    for (int c = 0; c < r; ++c) {
      double acc = 0;
      for (int j = 0; j < ns; ++j) acc += H[(size_t)i * ld + j] * F[(size_t)j * r + c];
      HF[(size_t)i * r + c] = acc;
    }
  for (int a2 = 0; a2 < r; ++a2)
    for (int c = 0; c < r; ++c) {
      double acc = 0;
      for (int i = 0; i < ns; ++i) acc += F[(size_t)i * r + a2] * HF[(size_t)i * r + c];
      Hr[(size_t)a2 * r + c] = acc;
    }
  std::vector<double> th, Y;
  if (r > 0) host_sym_eig(r, Hr, th, Y);
  std::vector<int> order(r);
  for (int i = 0; i < r; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return th[x] > th[y]; });
  for (int i = 0; i < ld * ld; ++i) C[i] = 0.0;
  for (int c = 0; c < kout; ++c) {
    if (c >= r) {
      theta[c] = -1.0;
      continue;
    }
    theta[c] = th[order[c]];
    for (int i = 0; i < ns; ++i) {
      double acc = 0;
      for (int a2 = 0; a2 < r; ++a2) acc += F[(size_t)i * r + a2] * Y[(size_t)a2 * r + order[c]];
      C[(size_t)i * ld + c] = acc;
    }
  }
}

void general_rr_batch(int nsub, int ns, int ld, int kout, const double *H, const double *M,
                      double *theta, double *C, int nthreads) {
  int nt = nthreads;
  if (nt <= 0) nt = (int)std::min<unsigned>(64, std::max(1u, std::thread::hardware_concurrency()));
  nt = std::max(1, std::min(nt, nsub));
  const size_t blk = (size_t)ld * ld;
  auto one = [&](int m) {
    general_rr(ns, ld, kout, H + m * blk, M + m * blk, theta + (size_t)m * kout, C + m * blk);
  };
  if (nt == 1) {
    for (int m = 0; m < nsub; ++m) one(m);
    return;
  }
  // subdomains handed out one at a time (their costs differ with the rank)
  std::atomic<int> next{0};
  std::vector<std::thread> th;
  th.reserve(nt);
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&]() {
      for (int m = next++; m < nsub; m = next++) one(m);
    });
  for (auto &x : th) x.join();
}

}  // namespace geneo
