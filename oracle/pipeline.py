"""End-to-end oracle set-up for one workload: mesh, assembly, decomposition,
coarse space (variants of Sec. 4: none / NK / SNK, with or without GenEO),
preconditioner and PCG."""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

from .mesh import build_mesh
from .fem import assemble_A, assemble_rhs, local_element_A
from .dd import decompose
from .coarse import (snk_columns, nk_columns, geneo_columns, assemble_Z, tau_paper,
                     independent_geneo, coarse_matrix)
from .solver import build_preconditioner, pcg


@dataclass
class OracleProblem:
    w: object
    mesh: object
    A: object
    AT: np.ndarray
    b: np.ndarray             # [nrhs, n]
    dec: object
    snk: list
    geneo: list
    gevps: list
    Z: object
    M: object
    tau_p: float
    info: dict = field(default_factory=dict)


def build_problem(w, *, coarse="snk", geneo=True, tau_convention="reciprocal",
                  pou="boolean", pencil="filtered"):
    mesh = build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active,
                      natural=getattr(w, "natural", None))
    A = assemble_A(mesh, w)
    AT = local_element_A(mesh, w)
    b = assemble_rhs(mesh, w)
    dec = decompose(mesh, w.parts, w.overlap, pou=pou)
    n = A.shape[0]
    if coarse == "snk":
        cols = snk_columns(mesh, dec)
    elif coarse == "nk":
        cols = nk_columns(mesh)
    elif coarse == "none":
        cols = []
    else:
        raise ValueError(coarse)
    tp = tau_paper(w.tau, tau_convention)
    gcols, gevps = ([], None)
    E = None
    if geneo:
        gcols, gevps = geneo_columns(mesh, w, A, AT, dec, tp, pencil=pencil)
        if gcols:
            E = coarse_matrix(mesh, w, assemble_Z(n, cols + gcols))
            keep = independent_geneo(E, len(cols))
            sel = np.concatenate([np.arange(len(cols)), len(cols) + keep])
            E = E[np.ix_(sel, sel)] if not hasattr(E, "tocsr") else E.tocsr()[sel][:, sel]
            gcols = [gcols[k] for k in keep.tolist()]
    Z = assemble_Z(n, cols + gcols) if (cols or gcols) else None
    if Z is not None and E is None:
        E = coarse_matrix(mesh, w, Z)
    M = build_preconditioner(A, dec, Z, E=E)
    return OracleProblem(w, mesh, A, AT, b, dec, cols, gcols, gevps, Z, M, tp)


def solve(prob, tol=1e-8, maxit=1000, rhs=0, balanced=False):
    """PCG with M^-1_AS,2; balanced=True starts from x0 = Z E^-1 Z^T b and
    applies the one-coarse-solve form (TwoLevel.apply_balanced)."""
    b = prob.b[rhs]
    if balanced and prob.M.Z is not None:
        return pcg(prob.A, b, prob.M.apply_balanced, tol=tol, maxit=maxit,
                   x0=prob.M.balanced_start(b))
    return pcg(prob.A, b, prob.M.apply, tol=tol, maxit=maxit)
