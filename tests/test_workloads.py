"""The seeded input generators follow their stated recipes (shapes, value
sets and ranges, partitions), so the parity and bench inputs stand for the
workloads they are named after."""
import numpy as np

import workloads as W


def test_batching_recipe():
    ps = W.many_problems(256, seed=3)
    assert len(ps) == 256
    for w in ps:
        n = w.nx
        assert w.ny == n and w.nz == n and 8 <= n <= 24
        assert abs(w.hx - 1.0 / n) < 1e-15
        assert 1e-6 <= w.gamma <= 1.0
        px, py, pz = w.parts
        assert {px, py, pz} <= {2, 3, 4} and 8 <= px * py * pz <= 64
        assert set(np.unique(w.mu_inv).tolist()) <= {1.0, 1e2, 1e4}
        act = w.active.reshape(n, n, n)
        holes = np.argwhere(act == 0)
        assert len(holes) > 0
        # holes stay one cell away from the outer boundary
        assert holes.min() >= 1 and holes.max() <= n - 2
    # seeded: the same draw twice
    again = W.many_problems(4, seed=3)
    assert all(np.array_equal(a.active, b.active) and a.gamma == b.gamma
               for a, b in zip(ps[:4], again))


def test_named_workloads_shapes():
    w = W.unit_cube_8()
    assert (w.nx, w.ny, w.nz, w.parts, w.overlap) == (8, 8, 8, (2, 2, 2), 1)
    assert w.gamma == 1.0 and np.all(w.mu_inv == 1.0) and np.all(w.active == 1)
    b = W.beam128_layered()
    assert (b.nx, b.ny, b.nz, b.parts, b.nrhs) == (128, 16, 16, (32, 4, 4), 16)
    assert b.gamma == 1e-6
    assert set(np.unique(b.mu_inv).tolist()) == {1.0, 1e6}
    c = W.cube32_hole_channels()
    assert (c.nx, c.ny, c.nz, c.parts, c.overlap) == (32, 32, 32, (4, 4, 4), 2)
    assert c.active.sum() == 32 ** 3 - 8 * 8 * 32
    assert 1.0 <= c.mu_inv.min() and c.mu_inv.max() <= 1e3
