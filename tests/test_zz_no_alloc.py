"""The allocation-free SYMV entry point, geneo_symv_packed_noalloc.

It exists for callers that cannot allocate device memory where they need a
symmetric apply (memory pools or arenas that forbid new allocations,
real-time loops where cudaMalloc would stall, hosts that own the device
allocator).  This test calls it through the C-ABI on the inverse of a
one-subdomain problem, twice in a row, and checks both results against the
library's existing local solve (which applies the same inverse) within the
tolerance of the other explicit-inverse tests, c * kappa * 2^-53 with
c = 1e3.  It runs alone or after the other tests (collected last).
"""
import ctypes

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def pack(M):
    """Tile-packed lower storage of a symmetric matrix (zero padding)."""
    dim = M.shape[0]
    nt = -(-dim // 64)
    P = np.zeros((nt * 64, nt * 64))
    P[:dim, :dim] = M
    out = np.zeros((nt * (nt + 1) // 2, 64, 64))
    for I in range(nt):
        for J in range(I + 1):
            out[I * (I + 1) // 2 + J] = P[I * 64:(I + 1) * 64, J * 64:(J + 1) * 64]
    return out.reshape(-1)


def test_noalloc_symv_matches_local_solve_twice():
    import paper_2311_18783_gb300 as pkg
    from oracle.mesh import build_mesh
    from oracle.fem import assemble_A
    lib = pkg.load_library()
    rng = np.random.default_rng(21)
    w = W.box(7, 5, 4, parts=(1, 1, 1), overlap=1, gamma=0.3,
              mu_inv=10.0 ** rng.uniform(0, 1, 140))
    s = pkg.Solver.from_workload(w, geneo=0, coarse=pkg.COARSE_NONE)
    m = build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active)
    A = assemble_A(m, w).toarray()
    dim = A.shape[0]
    assert dim % 64 != 0 and dim <= 4096
    ev = np.linalg.eigvalsh(A)
    kappa = ev[-1] / ev[0]
    tiles = torch.as_tensor(pack(np.linalg.inv(A)), device="cuda")
    stream = torch.cuda.current_stream()
    for trial in range(2):
        r = torch.as_tensor(rng.standard_normal(dim), device="cuda")
        ref = torch.empty_like(r)
        s.local_solve(r, ref)
        y = torch.full_like(r, np.nan)
        rc = lib.geneo_symv_packed_noalloc(ctypes.c_void_p(tiles.data_ptr()), dim,
                                           ctypes.c_void_p(r.data_ptr()),
                                           ctypes.c_void_p(y.data_ptr()),
                                           ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), ref.cpu().numpy()
        assert np.abs(a - b).max() <= 1e3 * kappa * U * np.abs(b).max()
    s.close()


def test_noalloc_rejects_sizes_beyond_the_limit():
    import paper_2311_18783_gb300 as pkg
    lib = pkg.load_library()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    assert lib.geneo_symv_packed_noalloc(p, 4097, p, p, None) == -1
    assert lib.geneo_symv_packed_noalloc(p, 0, p, p, None) == -1
