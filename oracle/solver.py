"""Two-level additive Schwarz preconditioner and PCG of the oracle.

M^-1_AS,2 = Z E^-1 Z^T + (I - P0) sum_i R_i^T A_i^-1 R_i (I - P0^T),
P0 = Z E^-1 Z^T A  (Sec. 2, eq. "AS2"; closed form at the end of Sec. 3.2),
applied in four literal steps:
    y0 = Z E^-1 Z^T r
    s  = r - A y0                      ((I - P0^T) r)
    w  = sum_i R_i^T A_i^-1 R_i s       (eq. "AS", Dirichlet A_i, no D_i)
    z  = y0 + w - Z E^-1 Z^T (A w)      (y0 + (I - P0) w)

PCG: M^-1 is symmetric (eq. "AS2") and A is SPD (Sec. 2), so the
preconditioned conjugate gradient applies; x0 = 0, stop when
||r_k||_2 / ||b||_2 <= tol on the recurrence residual.
"""
from __future__ import annotations

from dataclasses import dataclass
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


@dataclass
class TwoLevel:
    A: sp.csr_matrix
    N: list                 # restriction index sets
    Ainv_fact: list         # Cholesky factors of A_i (scipy cho_factor)
    Z: object               # sparse n x n0 (or None for one level)
    E_fact: object          # factor of E

    def coarse(self, v):
        if self.Z is None or self.Z.shape[1] == 0:
            return np.zeros_like(v)
        c = self.Z.T @ v
        y = self.E_fact(c)
        return self.Z @ y

    def local(self, s):
        w = np.zeros_like(s)
        for Ni, F in zip(self.N, self.Ainv_fact):
            w[Ni] += F(s[Ni])
        return w

    def apply(self, r):
        y0 = self.coarse(r)
        s = r - self.A @ y0
        w = self.local(s)
        return y0 + w - self.coarse(self.A @ w)

    # Balanced form (one coarse solve per apply).  If Z^T r = 0, the closed
    # form of M^-1_AS,2 (end of Sec. 3.2) loses its first term, Z E^-1 Z^T r,
    # and (I - P0^T) r = r - A Z E^-1 Z^T r = r, leaving (I - P0) M_loc r.
    # PCG started from x0 = Z E^-1 Z^T b has Z^T r_0 = Z^T b - E E^-1 Z^T b
    # = 0, and every later search direction lies in range(I - P0), on which
    # Z^T A vanishes (Z^T A (I - P0) = Z^T A - E E^-1 Z^T A = 0), so
    # Z^T r_k = 0 for every k in exact arithmetic.  In floating point Z^T r_k
    # drifts, and (I - P0) M_loc alone never corrects that drift (its
    # iterates stall above tight tolerances), so the apply adds back
    # Z E^-1 Z^T r, which is zero in exact arithmetic:
    #   z = w - Z E^-1 Z^T A w + Z E^-1 Z^T r = w + Z E^-1 Z^T (r - A w),
    # one coarse solve per apply (the "A-DEF2" two-level form of Tang,
    # Nabben, Vuik and Erlangga, J. Sci. Comput. 39, 2009).

    def balanced_start(self, b):
        """x0 = Z E^-1 Z^T b."""
        return self.coarse(b)

    def apply_balanced(self, r):
        """w + Z E^-1 Z^T (r - A w) with w = sum_i R_i^T A_i^-1 R_i r; equal
        to apply(r) when Z^T r = 0."""
        w = self.local(r)
        return w + self.coarse(r - self.A @ w)


def factor_dense(E):
    """Dense Cholesky (library primitive); returns the solve."""
    F = sla.cho_factor(E, lower=True)
    return lambda c: sla.cho_solve(F, c)


def factor_sparse(E):
    """Sparse LU (library primitive) for large SPD blocks; returns the solve."""
    lu = spla.splu(sp.csc_matrix(E))
    return lu.solve


def build_preconditioner(A, dec, Z, local_mats=None, E=None):
    """Local Cholesky factors of A_i and the factor of E = Z^T A Z (computed
    from the assembled A unless given)."""
    Ainv = []
    for i in range(dec.nsub):
        Ni = dec.N[i]
        if local_mats is not None:
            Ainv.append(factor_dense(local_mats[i]))
        elif len(Ni) <= 2000:
            Ainv.append(factor_dense(A[Ni][:, Ni].toarray()))
        else:
            Ainv.append(factor_sparse(A[Ni][:, Ni]))
    if Z is None or Z.shape[1] == 0:
        return TwoLevel(A, dec.N, Ainv, None, None)
    if E is None:
        E = (Z.T @ (A @ Z))
        E = E.toarray() if sp.issparse(E) else E
        E = 0.5 * (E + E.T)
    fact = factor_dense(E) if not sp.issparse(E) else factor_sparse(E)
    return TwoLevel(A, dec.N, Ainv, Z, fact)


@dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    relres: float
    history: list


def pcg(A, b, Minv, tol=1e-8, maxit=1000, x0=None):
    """Preconditioned CG from x0 (default 0); the stopping test is
    ||r_k|| <= tol ||b|| on the recurrence residual."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b.copy() if x0 is None else b - A @ x
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return PCGResult(np.zeros_like(b), 0, 0.0, [0.0])
    z = Minv(r)
    p = z.copy()
    rz = r @ z
    hist = [np.linalg.norm(r) / nb]
    for k in range(1, maxit + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        rel = np.linalg.norm(r) / nb
        hist.append(rel)
        if rel <= tol:
            return PCGResult(x, k, rel, hist)
        z = Minv(r)
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return PCGResult(x, maxit, hist[-1], hist)


def gmres_right(A, b, Minv, tol=1e-6, maxit=1000, restart=100):
    """Right-preconditioned restarted GMRES from x0 = 0 (Sec. 4: the paper's
    Krylov method): x_k = x0 + M^-1 V_k y_k with y_k minimising
    ||beta e_1 - H_k y|| over the Arnoldi basis V_k of A M^-1 (modified
    Gram-Schmidt, Givens rotations).  Stops when the true-residual estimate
    |g_{k+1}| <= tol ||b||, confirmed on b - A x at the end of a cycle.
    Returns PCGResult (iters = Arnoldi steps)."""
    n = b.shape[0]
    x = np.zeros(n)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return PCGResult(x, 0, 0.0, [0.0])
    its, hist = 0, []
    while its < maxit:
        r = b - A @ x
        beta = np.linalg.norm(r)
        hist.append(beta / nb)
        if beta <= tol * nb:
            return PCGResult(x, its, beta / nb, hist)
        m = restart
        V = np.zeros((m + 1, n))
        Zs = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        V[0] = r / beta
        g = np.zeros(m + 1)
        g[0] = beta
        cs, sn = np.zeros(m), np.zeros(m)
        k = 0
        for j in range(m):
            if its >= maxit:
                break
            Zs[j] = Minv(V[j])
            w = A @ Zs[j]
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                a, c = H[i, j], H[i + 1, j]
                H[i, j], H[i + 1, j] = cs[i] * a + sn[i] * c, -sn[i] * a + cs[i] * c
            rho = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / rho, H[j + 1, j] / rho
            H[j, j], H[j + 1, j] = rho, 0.0
            g[j + 1], g[j] = -sn[j] * g[j], cs[j] * g[j]
            its += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / nb)
            if abs(g[j + 1]) <= tol * nb:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + Zs[:k].T @ y
        if abs(g[k]) <= tol * nb:
            rel = np.linalg.norm(b - A @ x) / nb
            if rel <= tol or its >= maxit:
                return PCGResult(x, its, rel, hist)
    return PCGResult(x, its, np.linalg.norm(b - A @ x) / nb, hist)


def direct_solve(A, b):
    return spla.spsolve(sp.csc_matrix(A), b)


def residual_extended(A, b, x):
    """b - A x with every product and sum in numpy.longdouble (64-bit or
    113-bit significand, against float64's 53), returned in longdouble."""
    A = sp.csr_matrix(A)
    ld = np.longdouble
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    acc = np.zeros(A.shape[0], dtype=ld)
    np.add.at(acc, rows, A.data.astype(ld) * np.asarray(x, dtype=ld)[A.indices])
    return np.asarray(b, dtype=ld) - acc


def refined_direct_solve(A, b, steps=3):
    """x = A^-1 b by a sparse LU (library primitive; symmetric mode, minimum
    degree ordering on A + A^T) followed by `steps` rounds of classical
    iterative refinement with residuals in extended precision (Wilkinson):
    x <- x + LU^-1 (b - A x).  The float64 residual of any float64 x is
    bounded below by about u ||A|| ||x||, which bounds the forward error of
    plain float64 solves when A is ill conditioned (small gamma, Sec. 1);
    the extended residual removes that floor.  Returns (x, relative size of
    each correction)."""
    lu = spla.splu(sp.csc_matrix(A), permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                   options=dict(SymmetricMode=True))
    x = lu.solve(np.asarray(b, dtype=np.float64))
    hist = []
    for _ in range(steps):
        r = residual_extended(A, b, x).astype(np.float64)
        d = lu.solve(r)
        x = x + d
        hist.append(float(np.linalg.norm(d) / max(np.linalg.norm(x), 1e-300)))
    return x, hist
