"""Gradient shift of the local matrices: A~_j = A_j (I + rho xi_j) is inverted
instead of A_j, and A_j^-1 = A~_j^-1 + rho/(1+rho) G S^-1 G^T,
C_j = A~_j^-1 - 1/(1+rho) G S^-1 G^T hold exactly (xi_j a projection,
Sec. 2, lemma with eq. "inverseBw").

* Well-conditioned case: the shifted float64 and split local solves match the
  oracle's A_j^-1 within the same kappa(A_j) u bound as the unshifted ones, and
  PCG reaches the same solution in the same number of iterations.
* gamma = 1e-6 and a layered mu^-1 (kappa(A_j) up to ~1e16, beyond float64):
  with the shift, set-up succeeds and PCG converges to 1e-8 in the
  recurrence with float64 local factors under a 1e6 jump of mu^-1, with the
  float32 split under a 1e3 jump and with the bfloat16 split without a jump.
  (Measured: the rounded C_j turns indefinite once its rounding exceeds its
  smallest eigenvalues; float32 diverges at a 1e6 jump, bfloat16 at 1e3.)
  Here x carries gradients of size ~1/gamma that the curl part annihilates
  only in exact arithmetic, so no assembled product evaluates b - A x below
  the rounding floor u ||A| |x|| / ||b|| (about 0.4 for the oracle's own
  direct solution of such a case); the true residual, evaluated by the
  oracle on the host, must sit at that floor (within a factor 4).
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _pkg():
    import paper_2311_18783_gb300 as pkg
    pkg.load_library()
    return pkg


@pytest.fixture(scope="module")
def mild():
    from oracle.pipeline import build_problem
    from test_gpu_parity import hetero_box
    pkg = _pkg()
    w = hetero_box(seed=13)
    prob = build_problem(w, geneo=False)
    s0 = pkg.Solver.from_workload(w, geneo=0, precision=pkg.PREC_FP32)
    s1 = pkg.Solver.from_workload(w, geneo=0, precision=pkg.PREC_FP32, gradient_shift=1)
    yield pkg, w, prob, s0, s1
    s0.close()
    s1.close()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_shifted_local_solve(mild, prec):
    from test_gpu_parity import _kappa_local
    pkg, w, prob, s0, s1 = mild
    p = pkg.PREC_FP64 if prec == "fp64" else pkg.PREC_FP32
    r = np.random.default_rng(3).standard_normal(s1.n)
    ref = prob.M.local(r)
    tol = 1e3 * _kappa_local(prob) * U + (0.0 if prec == "fp64" else 1e-5)
    for s in (s0, s1):
        s.use_precision(p)
        out = torch.empty(s.n, dtype=torch.float64, device="cuda")
        s.local_solve(torch.as_tensor(r, device="cuda"), out)
        torch.cuda.synchronize()
        assert rel(out.cpu().numpy(), ref) <= tol


def test_shifted_pcg(mild):
    pkg, w, prob, s0, s1 = mild
    out = []
    for s in (s0, s1):
        s.use_precision(pkg.PREC_FP64)
        b = torch.empty(s.n, dtype=torch.float64, device="cuda")
        s.assemble_rhs(w.f_slot[0], b)
        x = torch.zeros_like(b)
        info = s.solve(b, x, tol=1e-10, maxit=500)
        assert info["status"] == 0
        out.append((x, info))
    (x0, i0), (x1, i1) = out
    assert abs(i0["iters"] - i1["iters"]) <= 1
    assert (torch.linalg.norm(x1 - x0) / torch.linalg.norm(x0)).item() <= 1e-8


def _layered_beam(contrast):
    # 32 x 4 x 4 cells, mu^-1 alternating 1 and `contrast` every 8 cells,
    # gamma 1e-6, boxes of 4 cells along x (the layering of the
    # 16-right-hand-side beam)
    nx, ny, nz = 32, 4, 4
    ci = np.arange(nx * ny * nz) % nx
    mu = np.where((ci // 8) % 2 == 0, 1.0, contrast)
    return W.box(nx, ny, nz, h=1 / 16, parts=(8, 1, 1), overlap=1, gamma=1e-6, mu_inv=mu,
                 f='random', seed=17)


@pytest.mark.parametrize("prec,contrast", [("fp64", 1e6), ("fp32", 1e3), ("bf16", 1.0)])
def test_shift_makes_tiny_gamma_solvable(prec, contrast):
    from oracle.mesh import build_mesh
    from oracle.fem import assemble_A, assemble_rhs
    pkg = _pkg()
    w = _layered_beam(contrast)
    s = pkg.Solver.from_workload(w, precision=pkg.PREC_BF16, gradient_shift=1)
    s.use_precision({"fp64": pkg.PREC_FP64, "fp32": pkg.PREC_FP32, "bf16": pkg.PREC_BF16}[prec])
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(w.f_slot[0], b)
    x = torch.zeros_like(b)
    info = s.solve(b, x, tol=1e-8, maxit=1000)
    s.close()
    assert info["status"] == 0
    m = build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active)
    A = assemble_A(m, w)
    bh = assemble_rhs(m, w)[0]
    xh = x.cpu().numpy()
    res = np.linalg.norm(bh - A @ xh) / np.linalg.norm(bh)
    floor = U * np.linalg.norm(abs(A) @ np.abs(xh)) / np.linalg.norm(bh)
    print(f"{prec}: {info['iters']} iterations, true relative residual {res:.2e}, "
          f"rounding floor {floor:.2e}")
    assert info["relres"] <= 1e-8
    assert res <= 4 * floor + 1e-7
