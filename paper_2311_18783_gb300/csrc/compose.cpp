// Composition of independent problems into one grid (see compose.hpp).
#include "compose.hpp"

#include <algorithm>
#include <string>

namespace geneo {

namespace {
void bad(const std::string &m) { throw Error(GENEO_ERR_INVALID_ARG, m); }
}  // namespace

void compose_problems(int32_t nprob, const geneo_problem *probs, bool arrays, Composite &out) {
  if (nprob < 1 || !probs) bad("compose: need at least one problem");
  out = Composite();
  double h = 0;
  int64_t z = 0;
  for (int32_t p = 0; p < nprob; ++p) {
    const geneo_problem &q = probs[p];
    if (q.nx < 1 || q.ny < 1 || q.nz < 1) bad("compose: grid sizes must be positive");
    if (!(q.hx > 0) || q.hx != q.hy || q.hx != q.hz) bad("compose: cells must be cubic");
    if (q.natural_faces) bad("compose: natural boundary faces are not supported");
    if (!(q.gamma > 0)) bad("compose: gamma must be > 0");
    if (q.overlap != probs[0].overlap || q.tau != probs[0].tau)
      bad("compose: all problems must share overlap and tau");
    if (!q.cell_part &&
        (q.px < 1 || q.py < 1 || q.pz < 1 || q.px > q.nx || q.py > q.ny || q.pz > q.nz))
      bad("compose: box counts must lie in [1, cells per axis]");
    if (arrays && (!q.active || !q.mu_inv || !q.eps)) bad("compose: null array");
    h = (p == 0) ? q.hx : std::min(h, q.hx);
    out.nx = std::max(out.nx, q.nx);
    out.ny = std::max(out.ny, q.ny);
    out.zoff.push_back((int32_t)z);
    z += q.nz + 1;
    if (z > (int64_t)1 << 30) bad("compose: composite too tall");
  }
  out.nz = (int32_t)(z - 1);
  out.h = h;
  const int64_t nc = (int64_t)out.nx * out.ny * out.nz;
  if (nc > (int64_t)1 << 28) bad("compose: composite mesh too large for int32 indices");
  if (!arrays) return;
  out.active.assign(nc, 0);
  out.mu_inv.assign(nc, 1.0);
  out.eps.assign(nc, 1.0);
  out.part.assign(nc, 0);
  int64_t pbase = 0;
  for (int32_t p = 0; p < nprob; ++p) {
    const geneo_problem &q = probs[p];
    const double r = q.hx / h;
    int64_t pmax = -1;
    for (int32_t k = 0; k < q.nz; ++k)
      for (int32_t j = 0; j < q.ny; ++j)
        for (int32_t i = 0; i < q.nx; ++i) {
          const int64_t c = i + (int64_t)q.nx * (j + (int64_t)q.ny * k);
          const int64_t g = i + (int64_t)out.nx * (j + (int64_t)out.ny * (k + out.zoff[p]));
          out.active[g] = q.active[c] ? 1 : 0;
          out.mu_inv[g] = q.mu_inv[c] / r;
          out.eps[g] = q.eps[c] * q.gamma * r;
          int64_t part;
          if (q.cell_part) {
            part = q.cell_part[c];
            if (q.active[c] && part < 0) bad("compose: cell_part must be >= 0 on active cells");
            if (!q.active[c]) part = 0;
          } else {
            part = (int64_t)i * q.px / q.nx +
                   (int64_t)q.px * ((int64_t)j * q.py / q.ny + (int64_t)q.py * ((int64_t)k * q.pz / q.nz));
          }
          if (q.active[c]) pmax = std::max(pmax, part);
          part += pbase;
          if (part >= (1 << 24)) bad("compose: more than 2^24 subdomains");
          out.part[g] = (int32_t)part;
        }
    pbase += q.cell_part ? pmax + 1 : (int64_t)q.px * q.py * q.pz;
  }
}

void compose_field(int32_t nprob, const geneo_problem *probs, const Composite &cmp,
                   const double *const *f_slot, int32_t nrhs, double *out) {
  if (nrhs < 1 || !out) bad("compose: nrhs >= 1 and an output array are required");
  const int64_t nv = (int64_t)(cmp.nx + 1) * (cmp.ny + 1) * (cmp.nz + 1);
  std::fill(out, out + (size_t)nrhs * nv * 21, 0.0);
  for (int32_t p = 0; p < nprob; ++p) {
    if (!f_slot || !f_slot[p]) continue;
    const geneo_problem &q = probs[p];
    const double r = q.hx / cmp.h, s = r * r;
    const int64_t nvp = (int64_t)(q.nx + 1) * (q.ny + 1) * (q.nz + 1);
    for (int32_t rhs = 0; rhs < nrhs; ++rhs)
      for (int32_t k = 0; k <= q.nz; ++k)
        for (int32_t j = 0; j <= q.ny; ++j)
          for (int32_t i = 0; i <= q.nx; ++i) {
            const int64_t v = i + (int64_t)(q.nx + 1) * (j + (int64_t)(q.ny + 1) * k);
            const int64_t g =
                i + (int64_t)(cmp.nx + 1) * (j + (int64_t)(cmp.ny + 1) * (k + cmp.zoff[p]));
            const double *src = f_slot[p] + ((size_t)rhs * nvp + v) * 21;
            double *dst = out + ((size_t)rhs * nv + g) * 21;
            for (int e = 0; e < 21; ++e) dst[e] = src[e] * s;
          }
  }
}

}  // namespace geneo
