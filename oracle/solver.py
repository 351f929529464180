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


def pcg(A, b, Minv, tol=1e-8, maxit=1000):
    """Preconditioned CG from x0 = 0."""
    x = np.zeros_like(b)
    r = b.copy()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return PCGResult(x, 0, 0.0, [0.0])
    z = Minv(r)
    p = z.copy()
    rz = r @ z
    hist = [1.0]
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


def direct_solve(A, b):
    return spla.spsolve(sp.csc_matrix(A), b)
