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


def test_noalloc_symv_at_the_size_limit_matches_numpy():
    """dim = 4096, the largest size the fixed scratch array holds (64 tiles
    per side, every column-partial slot used), on a random symmetric matrix,
    two calls in a row.  Reference: NumPy's float64 product T @ x on the
    host.  Both sums have at most dim terms, so each side is within
    dim * u * (|T| |x|) of the exact product (the standard bound for a dot
    product in floating point); the test allows 64 dim u (|T| |x|)."""
    import paper_2311_18783_gb300 as pkg
    lib = pkg.load_library()
    rng = np.random.default_rng(33)
    dim = 4096
    T = rng.standard_normal((dim, dim))
    T = 0.5 * (T + T.T)
    tiles = torch.as_tensor(pack(T), device="cuda")
    stream = torch.cuda.current_stream()
    for trial in range(2):
        x = rng.standard_normal(dim)
        xd = torch.as_tensor(x, device="cuda")
        y = torch.full_like(xd, np.nan)
        rc = lib.geneo_symv_packed_noalloc(ctypes.c_void_p(tiles.data_ptr()), dim,
                                           ctypes.c_void_p(xd.data_ptr()),
                                           ctypes.c_void_p(y.data_ptr()),
                                           ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        ref = T @ x
        bound = 64 * dim * U * (np.abs(T) @ np.abs(x))
        assert np.all(np.abs(y.cpu().numpy() - ref) <= bound)


def test_noalloc_rejects_sizes_beyond_the_limit():
    import paper_2311_18783_gb300 as pkg
    lib = pkg.load_library()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    assert lib.geneo_symv_packed_noalloc(p, 4097, p, p, None) == -1
    assert lib.geneo_symv_packed_noalloc(p, 0, p, p, None) == -1


def test_noalloc_rejects_misaligned_tiles():
    """The tiles are read by bulk copies from 16-byte aligned addresses
    only: a pointer 8 bytes past an aligned one is refused with INVALID_ARG
    before any launch."""
    import paper_2311_18783_gb300 as pkg
    lib = pkg.load_library()
    t = torch.zeros(2 * 4096 + 2, dtype=torch.float64, device="cuda")
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    y = torch.zeros(64, dtype=torch.float64, device="cuda")
    assert t.data_ptr() % 16 == 0
    rc = lib.geneo_symv_packed_noalloc(ctypes.c_void_p(t.data_ptr() + 8), 64,
                                       ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(y.data_ptr()), None)
    assert rc == -1
