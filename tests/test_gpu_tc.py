"""Tensor-core local solves: the split local inverse with C_j = (I - xi_j) A_j^-1
in bfloat16 (Sec. 2, eq. "inverseBw"), applied by tcgen05 MMAs to blocks of
right-hand sides with float32 accumulation.

* Exactness of the kernel: y_bf16 - y_fp32 (the float64 gradient parts cancel)
  against the same difference emulated in float64 from the library's own
  float32 C_j rounded to bfloat16, applied in the two-sided form
  (I - xi_j) C_j (I - xi_j)^T x (equal to C_j x in exact arithmetic) to the
  residual rounded to bfloat16 after the right projection.  The remaining
  gap is float32 accumulation (<= n_j 2^-24 |C||x| per entry): bound
  1e-5 ||C||x|| + 5% of the difference itself.  A misplaced or mis-transposed
  tile gives an O(1) error.
* Precision: ||y_bf16 - y_fp32|| <= 2^-6 ||y_fp32||.
* Columns are independent: a block of 16 equals the single-column results.
* Block PCG with bfloat16 local factors converges to 1e-8; the solution is
  compared with the float64 solution.
* Subdomains above 2048 local unknowns are refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tcs():
    import paper_2311_18783_gb300 as pkg
    from test_gpu_parity import hetero_box
    w = hetero_box(seed=11)
    s = pkg.Solver.from_workload(w, precision=pkg.PREC_BF16)
    yield pkg, w, s
    s.close()


def _dense_C(s, i):
    """C_i (float32) from the library's tile-packed storage."""
    nt = s.export("loc_nt")
    toff = s.export("loc_toff")
    f32 = s.export("loc_f32").reshape(-1, 64, 64)
    n = int(nt[i]) * 64
    C = np.zeros((n, n), dtype=np.float32)
    for I in range(nt[i]):
        for J in range(I + 1):
            t = f32[toff[i] + I * (I + 1) // 2 + J]
            C[I * 64:(I + 1) * 64, J * 64:(J + 1) * 64] = t
            if I != J:
                C[J * 64:(J + 1) * 64, I * 64:(I + 1) * 64] = t.T
    return C


def _bf16(a):
    return torch.as_tensor(a).to(torch.bfloat16).to(torch.float64).numpy()


def test_tc_local_solve_exact(tcs):
    pkg, w, s = tcs
    r = np.random.default_rng(3).standard_normal(s.n)
    rd = torch.as_tensor(r, device="cuda")
    y16 = torch.empty_like(rd)
    y32 = torch.empty_like(rd)
    s.use_precision(pkg.PREC_BF16)
    s.local_solve(rd, y16)
    s.use_precision(pkg.PREC_FP32)
    s.local_solve(rd, y32)
    s.use_precision(pkg.PREC_BF16)
    d = (y16 - y32).cpu().numpy()
    from oracle.mesh import build_mesh
    from oracle.fem import assemble_A
    from oracle.dd import decompose
    from oracle.coarse import local_gradient, xi_projector
    mesh = build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active)
    A = assemble_A(mesh, w).tocsr()
    dec = decompose(mesh, w.parts, w.overlap)
    noff, nidx = s.export("N_off"), s.export("N_idx")
    dref = np.zeros(s.n)
    cx = np.zeros(s.n)
    for i in range(len(noff) - 1):
        idx = nidx[noff[i]:noff[i + 1]]
        assert np.array_equal(idx, dec.N[i])
        C = _dense_C(s, i)[:len(idx), :len(idx)].astype(np.float64)
        x = r[idx]
        Gi, _ = local_gradient(mesh, dec, i)
        xi = xi_projector(A[idx][:, idx].toarray(), Gi)
        xp = x - xi.T @ x
        v = _bf16(C) @ _bf16(xp)
        e = (v - xi @ v) - C @ x
        np.add.at(dref, idx, e)
        np.add.at(cx, idx, np.abs(C) @ np.abs(x))
    err = np.linalg.norm(d - dref)
    assert err <= 1e-5 * np.linalg.norm(cx) + 0.05 * np.linalg.norm(dref)
    y32h = y32.cpu().numpy()
    assert np.linalg.norm(d) <= 2.0 ** -6 * np.linalg.norm(y32h)


def test_tc_columns_independent(tcs):
    pkg, w, s = tcs
    s.use_precision(pkg.PREC_BF16)
    R = torch.as_tensor(np.random.default_rng(5).standard_normal((16, s.n)), device="cuda")
    Z = torch.empty_like(R)
    s.apply_preconditioner_block(R, Z)
    for j in (0, 7, 15):
        z = torch.empty_like(R[j])
        s.apply_preconditioner(R[j].contiguous(), z)
        assert torch.allclose(Z[j], z, rtol=1e-6, atol=1e-12 * z.abs().max().item())


def test_tc_block_pcg(tcs):
    pkg, w, s = tcs
    import dataclasses
    import workloads as W
    nverts = (w.nx + 1) * (w.ny + 1) * (w.nz + 1)
    f = W._uniform_f(np.random.default_rng(8), nverts, 4)
    B = torch.empty((4, s.n), dtype=torch.float64, device="cuda")
    for j in range(4):
        s.assemble_rhs(f[j], B[j])
    s.use_precision(pkg.PREC_FP64)
    X64 = torch.empty_like(B)
    st64, i64 = s.solve_block(B, X64, tol=1e-8, maxit=500)
    s.use_precision(pkg.PREC_BF16)
    X16 = torch.empty_like(B)
    st16, i16 = s.solve_block(B, X16, tol=1e-8, maxit=500)
    assert st64 == 0 and st16 == 0
    for j in range(4):
        assert i16[j]["relres"] <= 1e-8
        assert i16[j]["iters"] <= i64[j]["iters"] + 5
        d = (torch.linalg.norm(X16[j] - X64[j]) / torch.linalg.norm(X64[j])).item()
        print(f"rhs {j}: bf16 vs float64 solution {d:.2e}, iterations {i16[j]['iters']} vs "
              f"{i64[j]['iters']}")
        assert d <= 1e-5


def test_tc_refuses_large_subdomains():
    import paper_2311_18783_gb300 as pkg
    import workloads as W
    w = W.box(8, 8, 8, parts=(1, 1, 1), overlap=1)
    with pytest.raises(pkg.GeneoError):
        pkg.Solver.from_workload(w, precision=pkg.PREC_BF16, geneo=0)
