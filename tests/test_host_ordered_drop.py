"""GenEO independence filter on the host (csrc/ordered_drop.cpp, plain C++
with threads) compiled with g++:
* on the GenEO Schur complement of real coarse spaces, the kept columns equal
  the oracle's ordered Cholesky (oracle/coarse.py, independent_geneo);
* planted dependent columns (exact linear combinations of earlier ones) are
  the ones dropped;
* the pivots do not depend on the number of threads, bit for bit (every
  entry sees the same operations in the same order), across several panels."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2311_18783_gb300", "csrc")
P = C.POINTER(C.c_double)
TOL = 1e-8


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("ordered_drop")
    shim = d / "shim.cpp"
    shim.write_text(
        '#include <vector>\n#include "ordered_drop.hpp"\n'
        'extern "C" long drop(long nh, const double *S, const double *dg, double tol, int nt,\n'
        '                     long *keep, double *piv) {\n'
        '  std::vector<double> s(S, S + nh * nh), g(dg, dg + nh), p;\n'
        '  auto k = geneo::ordered_drop(s, g, nh, tol, nt, &p);\n'
        '  for (size_t i = 0; i < k.size(); ++i) keep[i] = k[i];\n'
        '  for (long i = 0; i < nh; ++i) piv[i] = p[i];\n'
        '  return (long)k.size();\n}\n')
    so = d / "ordered_drop.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-I" + SRC,
                    os.path.join(SRC, "ordered_drop.cpp"), str(shim), "-o", str(so)], check=True)
    return C.CDLL(str(so))


def _drop(lib, S, diag, nt=1):
    nh = S.shape[0]
    keep = np.zeros(nh, np.int64)
    piv = np.zeros(nh)
    S = np.ascontiguousarray(S, dtype=np.float64)
    diag = np.ascontiguousarray(diag, dtype=np.float64)
    lib.drop.restype = C.c_long
    k = lib.drop(C.c_long(nh), S.ctypes.data_as(P), diag.ctypes.data_as(P), C.c_double(TOL),
                 C.c_int(nt), keep.ctypes.data_as(C.POINTER(C.c_long)), piv.ctypes.data_as(P))
    return keep[:k], piv


def _schur(E, ns):
    import scipy.linalg as sla
    E = E.toarray() if hasattr(E, "toarray") else np.asarray(E)
    Ehh, Egh, Egg = E[ns:, ns:], E[:ns, ns:], E[:ns, :ns]
    S = Ehh - Egh.T @ sla.cho_solve(sla.cho_factor(Egg), Egh) if ns else Ehh
    return 0.5 * (S + S.T), np.diag(Ehh).copy()


def test_matches_oracle_on_a_coarse_space(lib):
    """A cube of the batching workload (n = 9, 16 boxes, holes, mu^-1 in
    {1, 1e2, 1e4}, gamma 4.2e-3): 68 GenEO candidates, of which the oracle
    keeps 66."""
    from oracle.pipeline import build_problem
    from oracle.coarse import (geneo_columns, snk_columns, coarse_matrix, assemble_Z,
                               independent_geneo)
    w = [w for w in W.many_problems(256, seed=3) if w.nx <= 10][2]
    prob = build_problem(w, geneo=False)
    cols = snk_columns(prob.mesh, prob.dec)
    gcols, _ = geneo_columns(prob.mesh, w, prob.A, prob.AT, prob.dec, prob.tau_p)
    assert len(gcols) > 0
    E = coarse_matrix(prob.mesh, w, assemble_Z(prob.A.shape[0], cols + gcols))
    ref = independent_geneo(E, len(cols))
    S, diag = _schur(E, len(cols))
    keep, _ = _drop(lib, S, diag)
    assert list(keep) == list(ref)
    assert len(gcols) == 68 and len(ref) == 66


def test_planted_dependence_and_thread_invariance(lib):
    rng = np.random.default_rng(3)
    n, m = 900, 700
    V = rng.standard_normal((n, m))
    dep = sorted(rng.choice(np.arange(5, m), 60, replace=False).tolist())
    for c in dep:  # exact combination of three earlier columns
        a, b, d = rng.choice(c, 3, replace=False)
        V[:, c] = V[:, a] - 2.0 * V[:, b] + 0.5 * V[:, d]
    S = V.T @ V
    k1, p1 = _drop(lib, S, np.diag(S), nt=1)
    k7, p7 = _drop(lib, S, np.diag(S), nt=7)
    assert np.array_equal(k1, k7)
    assert np.array_equal(p1, p7)
    assert sorted(set(range(m)) - set(k1.tolist())) == dep
