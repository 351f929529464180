"""The SYMV autotuner (options.autotune): every candidate launch
configuration of the streaming SYMV computes the same local solve (only the
association of the column partial sums differs: relative 1e-13 in float64,
1e-5 in float32 against the default configuration), the tuner records a
timing for every candidate and keeps the fastest, and a second set-up of the
same shapes takes the choice from the cache file without timing."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case():
    rng = np.random.default_rng(3)
    n = (10, 8, 6)
    nc = n[0] * n[1] * n[2]
    return W.box(*n, parts=(3, 2, 1), overlap=1, gamma=1e-2,
                 mu_inv=10.0 ** rng.uniform(0, 2, nc), f='random', seed=3, tau=0.1)


def test_every_configuration_same_local_solve():
    import paper_2311_18783_gb300 as pkg
    w = _case()
    s = pkg.Solver.from_workload(w, precision=pkg.PREC_FP32)
    r = torch.as_tensor(np.random.default_rng(0).standard_normal(s.n), device="cuda")
    for prec, tol in ((pkg.PREC_FP64, 1e-13), (pkg.PREC_FP32, 1e-5)):
        s.use_precision(prec)
        ref = torch.empty_like(r)
        s.use_symv_config(prec, 0)
        s.local_solve(r, ref)
        for i in range(1, pkg.Solver.symv_config_count(prec)):
            s.use_symv_config(prec, i)
            y = torch.empty_like(r)
            s.local_solve(r, y)
            d = (torch.linalg.norm(y - ref) / torch.linalg.norm(ref)).item()
            assert d <= tol, (prec, i, d)
            # the same configuration twice: bit for bit
            y2 = torch.empty_like(r)
            s.local_solve(r, y2)
            assert torch.equal(y, y2)
        s.use_symv_config(prec, 0)
    with pytest.raises(pkg.GeneoError):
        s.use_symv_config(pkg.PREC_FP64, 99)
    s.close()


def test_autotune_records_and_cache(tmp_path):
    import paper_2311_18783_gb300 as pkg
    w = _case()
    cache = str(tmp_path / "symv_tune.txt")
    s = pkg.Solver.from_workload(w, precision=pkg.PREC_FP32, autotune=1, autotune_cache=cache)
    rows = s.export("autotune").reshape(-1, 12)
    # local float32 and float64, S_j^-1 float64 and float32, coarse solve shape
    assert len(rows) == 5
    assert list(rows[:, 0]) == [0, 0, 1, 1, 2]
    for row in rows:
        prec = int(row[1])
        ncand = pkg.Solver.symv_config_count(prec) if row[0] < 2 else 2
        ms = row[4:4 + ncand]
        assert row[3] == 0 and np.all(ms > 0)
        assert np.all(np.isnan(row[4 + ncand:]))
        assert int(row[2]) == int(np.argmin(ms))
    stages = s.export("setup_stages")
    assert stages[6] > 0 and abs(stages[:7].sum() - stages[7]) <= 0.05 * stages[7] + 0.05
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(w.f_slot[0], b)
    x = torch.zeros_like(b)
    assert s.solve(b, x, tol=1e-10, maxit=500)["status"] == 0
    s.close()
    s2 = pkg.Solver.from_workload(w, precision=pkg.PREC_FP32, autotune=1, autotune_cache=cache)
    rows2 = s2.export("autotune").reshape(-1, 12)
    assert np.all(rows2[:, 3] == 1) and np.array_equal(rows2[:, 2], rows[:, 2])
    s2.close()


def test_four_column_pass_equals_columns_under_every_configuration():
    """A block apply of float32 local solves streams each tile once for four
    columns (k_symv_strips_nr); with the warps per tile of the selected
    configuration it keeps every sum in the single-column order, so each
    column of a 6-column block equals its own single-column apply bit for
    bit (columns 0-3 through the four-column kernel, 4-5 one at a time),
    under 8- and 16-warp configurations alike."""
    import paper_2311_18783_gb300 as pkg
    w = _case()
    s = pkg.Solver.from_workload(w, precision=pkg.PREC_FP32)
    s.use_precision(pkg.PREC_FP32)
    R = torch.as_tensor(np.random.default_rng(5).standard_normal((6, s.n)), device="cuda")
    for i in range(pkg.Solver.symv_config_count(pkg.PREC_FP32)):
        s.use_symv_config(pkg.PREC_FP32, i)
        Z = torch.empty_like(R)
        s.apply_preconditioner_block(R, Z)
        for j in range(6):
            z = torch.empty_like(R[j])
            s.apply_preconditioner(R[j].contiguous(), z)
            assert torch.equal(Z[j], z), (i, j)
    s.use_symv_config(pkg.PREC_FP32, 0)
    s.close()
