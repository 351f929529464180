// Small dense symmetric eigenproblems of the batched LOBPCG, on the host.
#pragma once
#include <vector>

namespace geneo {

// Cyclic Jacobi: a is n x n row-major (destroyed); w gets the eigenvalues,
// v (n x n, row-major) the eigenvectors as columns.
void host_sym_eig(int n, std::vector<double> &a, std::vector<double> &w, std::vector<double> &v);

// Rayleigh-Ritz of one subdomain in a basis S that is not B-orthonormal:
// H = S^T L S and M = S^T B S (ns x ns, leading dimension ld).  M = U E U^T,
// directions with E <= 1e-12 max(E) are dropped, F = U_keep E_keep^-1/2, and
// the standard problem F^T H F y = theta y gives the Ritz vectors S F y.
// Writes the kout largest theta and their coefficient columns C = F y
// (C[i * ld + c], ld x ld zero-filled); missing columns (rank below kout)
// get theta = -1 and C = 0.
void general_rr(int ns, int ld, int kout, const double *H, const double *M, double *theta,
                double *C);

// general_rr for nsub independent subdomains (H, M: nsub blocks of ld x ld;
// theta: nsub x kout; C: nsub blocks of ld x ld), spread over host threads
// (nthreads <= 0: the hardware concurrency, at most 64).  Each subdomain is
// computed by one thread with the code above, so the results do not depend
// on the number of threads.
void general_rr_batch(int nsub, int ns, int ld, int kout, const double *H, const double *M,
                      double *theta, double *C, int nthreads = 0);

}  // namespace geneo
