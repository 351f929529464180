"""Plain FP64 CPU oracle for the AS-SNK-GenEO preconditioned Krylov solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA library; the only
common module is ``workloads`` (seeded inputs, no method arithmetic).

It follows Bootland, Dolean, Nataf, Tournier, "A robust and adaptive
GenEO-type domain decomposition preconditioner for H(curl) problems in
three-dimensional general topologies" (arXiv 2311.18783):

* ``mesh``   structured Kuhn tetrahedra, edges, Dirichlet boundary, incidence
             matrices G (the gradient near-kernel of Sec. 1 and of the
             definition "near-kernelCS" in Sec. 2) and F;
* ``fem``    lowest-order Nedelec (Whitney) element matrices for the bilinear
             form of Sec. 2, eq. "bilinearformposmax", A = K + gamma*M of
             Sec. 1, eq. "discretemaxwell", and the load l(v);
* ``dd``     overlapping boxes, restriction sets N_i, the partition of unity
             of Sec. 2, eq. "PoU", k0 (eq. "k0") and k1, Dirichlet matrices
             A_i = R_i A R_i^T (eq. "AS") and Neumann matrices A_i^Neu;
* ``coarse`` the split near-kernel space (Sec. 2, definition
             "near-kernelCS"), the projection xi_0i (Sec. 2, lemma with
             eq. "inverseBw"), the filtered generalised eigenproblem (Sec. 3.2,
             GEVP "tauthresholdAS", eq. "eigAtildeBAS"), the GenEO selection
             lambda > tau, Z and E = Z^T A Z (eq. "V0GenEOAS");
* ``solver`` the two-level preconditioner M^-1_AS,2 (Sec. 2, eq. "AS2", and
             its closed form at the end of Sec. 3.2), preconditioned CG and a
             direct solve.

Every function states the passage it follows.  All floating point is
float64.  Where the paper is silent the oracle takes these readings: the
Kuhn six-tetrahedra split of each cubic cell, Dirichlet dofs eliminated, the
Boolean partition of unity (an edge belongs to the subdomain of the lowest
active cell containing it, D_i = 1 on the edges subdomain i owns; the
core-edge alternative D_i(e) = chi_i(e) / sum_j chi_j(e) is kept as
``decompose(..., pou="core")``), the reciprocal tau convention (select
lambda > 1/tau) by default, and removal of duplicate and floating
near-kernel columns so that Z has full rank.
"""
