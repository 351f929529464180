"""Host eigen-solvers of the batched LOBPCG (csrc/small_eig.cpp, plain C++)
compiled with g++ and checked against LAPACK through NumPy:
* host_sym_eig: eigenvalues and orthonormal eigenvectors of random
  symmetric matrices, including repeated eigenvalues;
* general_rr: the Rayleigh-Ritz step in a basis that is not B-orthonormal
  (used by the lobpcg_neumann mode) returns the kout largest eigenvalues of
  the pencil restricted to span S, B-orthonormal Ritz vectors, and a residual
  orthogonal to span S, also when S has a numerically dependent column;
* general_rr_batch: the same step for many subdomains over host threads
  equals the one-subdomain calls bit for bit, for any thread count."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2311_18783_gb300", "csrc")
P = C.POINTER(C.c_double)


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("small_eig")
    shim = d / "shim.cpp"
    shim.write_text(
        '#include <vector>\n#include "small_eig.hpp"\n'
        'extern "C" void eig(int n, const double *a, double *w, double *v) {\n'
        '  std::vector<double> A(a, a + (size_t)n * n), W, V;\n'
        '  geneo::host_sym_eig(n, A, W, V);\n'
        '  for (int i = 0; i < n; ++i) w[i] = W[i];\n'
        '  for (size_t i = 0; i < V.size(); ++i) v[i] = V[i];\n}\n'
        'extern "C" void rr(int ns, int ld, int k, const double *H, const double *M,\n'
        '                   double *th, double *Cm) { geneo::general_rr(ns, ld, k, H, M, th, Cm); }\n'
        'extern "C" void rr_batch(int nsub, int ns, int ld, int k, const double *H,\n'
        '                         const double *M, double *th, double *Cm, int nt) {\n'
        '  geneo::general_rr_batch(nsub, ns, ld, k, H, M, th, Cm, nt); }\n')
    so = d / "small_eig.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-I" + SRC,
                    os.path.join(SRC, "small_eig.cpp"), str(shim), "-o", str(so)], check=True)
    return C.CDLL(str(so))


def test_jacobi_matches_lapack(lib):
    rng = np.random.default_rng(0)
    for n in (1, 2, 7, 24, 48):
        A = rng.standard_normal((n, n))
        A = A + A.T
        if n >= 7:  # a repeated eigenvalue
            Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
            ev = rng.standard_normal(n)
            ev[1] = ev[0]
            A = Q @ np.diag(ev) @ Q.T
        w = np.zeros(n)
        V = np.zeros((n, n))
        lib.eig(n, np.ascontiguousarray(A).ctypes.data_as(P), w.ctypes.data_as(P),
                V.ctypes.data_as(P))
        ref = np.linalg.eigvalsh(A)
        assert np.abs(np.sort(w) - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())
        assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-13
        assert np.abs(A @ V - V * w).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_general_rayleigh_ritz(lib):
    rng = np.random.default_rng(1)
    ld, n = 64, 150
    for trial in range(12):
        ns = int(rng.choice([16, 24, 48]))
        k = ns // 3
        B = rng.standard_normal((n, n))
        B = B @ B.T / n + 1e-3 * np.eye(n)
        L = rng.standard_normal((n, n))
        L = L @ L.T * 10.0 ** rng.uniform(-2, 6)
        S = rng.standard_normal((n, ns))
        if trial % 3 == 0:
            S[:, -1] = S[:, 0] + 1e-14 * S[:, 1]
        H = np.zeros((ld, ld))
        M = np.zeros((ld, ld))
        H[:ns, :ns] = S.T @ L @ S
        M[:ns, :ns] = S.T @ B @ S
        th = np.zeros(k)
        Cm = np.zeros((ld, ld))
        lib.rr(ns, ld, k, H.ctypes.data_as(P), M.ctypes.data_as(P), th.ctypes.data_as(P),
               Cm.ctypes.data_as(P))
        # reference: the pencil on span S, computed from an orthonormal basis of S
        Qs, sv, _ = np.linalg.svd(S, full_matrices=False)
        Qs = Qs[:, sv > 1e-9 * sv[0]]
        ref = np.sort(np.linalg.eigvals(np.linalg.solve(Qs.T @ B @ Qs, Qs.T @ L @ Qs)).real)[::-1]
        assert np.abs(th - ref[:k]).max() <= 1e-9 * ref[0]
        assert np.all(np.diff(th) <= 0)
        X = S @ Cm[:ns, :k]
        assert np.abs(X.T @ B @ X - np.eye(k)).max() <= 1e-9
        R = L @ X - B @ X * th
        assert np.abs(S.T @ R).max() <= 1e-9 * np.abs(S.T @ L @ X).max()


def test_general_rr_batch_equals_single_calls(lib):
    rng = np.random.default_rng(17)
    nsub, ns, ld, k = 13, 24, 32, 8
    H = np.zeros((nsub, ld, ld))
    M = np.zeros((nsub, ld, ld))
    for m in range(nsub):
        S = rng.standard_normal((40, ns))
        if m % 4 == 0:
            S[:, 5] = S[:, 1] - 2.0 * S[:, 3]  # a dependent direction
        A = rng.standard_normal((40, 40))
        Bm = rng.standard_normal((40, 40))
        H[m, :ns, :ns] = S.T @ (A + A.T) @ S
        M[m, :ns, :ns] = S.T @ (Bm @ Bm.T + 40 * np.eye(40)) @ S
    th1 = np.zeros((nsub, k))
    C1 = np.zeros((nsub, ld, ld))
    for m in range(nsub):
        t = np.zeros(k)
        c = np.zeros((ld, ld))
        lib.rr(ns, ld, k, H[m].ctypes.data_as(P), M[m].ctypes.data_as(P),
               t.ctypes.data_as(P), c.ctypes.data_as(P))
        th1[m], C1[m] = t, c
    for nt in (1, 3, 8):
        th = np.zeros((nsub, k))
        Cb = np.zeros((nsub, ld, ld))
        lib.rr_batch(nsub, ns, ld, k, H.ctypes.data_as(P), M.ctypes.data_as(P),
                     th.ctypes.data_as(P), Cb.ctypes.data_as(P), nt)
        assert np.array_equal(th, th1) and np.array_equal(Cb, C1), nt
