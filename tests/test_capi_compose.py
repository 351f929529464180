"""Host-only composition of independent problems in the C-ABI
(geneo_compose*, no GPU needed) against workloads.compose, bit for bit:
the same arrays, offsets and composed load.  The composite's operator is
pinned to the separate problems' operators by test_compose_is_block_diagonal
(oracle), and the Python composition is the one the segmented GPU solve is
checked with."""
import os

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def pkg():
    from paper_2311_18783_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_2311_18783_gb300 as p
    p.load_library()
    return p


def _same(pkg, ps):
    ref = W.compose(ps)
    got = pkg.compose(ps)
    assert (got["nx"], got["ny"], got["nz"]) == (ref.nx, ref.ny, ref.nz)
    assert got["h"] == ref.hx
    assert list(got["zoff"]) == list(ref.meta["zoff"])
    assert np.array_equal(got["active"], ref.active)
    assert np.array_equal(got["cell_part"], ref.cell_part)
    assert np.array_equal(got["mu_inv"], ref.mu_inv)
    assert np.array_equal(got["eps"], ref.eps)
    assert np.array_equal(got["f_slot"], ref.f_slot)
    return got


def test_same_cell_size(pkg):
    rng = np.random.default_rng(5)
    ps = [W.box(6, 6, 6, h=1 / 6, parts=(2, 1, 1), gamma=1e-2,
                mu_inv=10.0 ** rng.uniform(0, 2, 216), f='random', seed=1),
          W.box(5, 4, 4, h=1 / 6, parts=(1, 2, 1), gamma=1.0, f='random', seed=2),
          W.box(4, 4, 3, h=1 / 6, parts=(2, 1, 1), gamma=0.5, f=(0.0, 0.0, 0.0))]
    got = _same(pkg, ps)
    assert sorted(set(got["cell_part"][got["active"] == 1].tolist())) == list(range(6))


def test_mixed_cell_sizes_and_holes(pkg):
    ps = [w for w in W.many_problems(256, seed=3) if w.nx <= 10][:5]
    for w in ps:
        w.f_slot = W.box(w.nx, w.ny, w.nz, h=w.hx, f='random', seed=w.nx).f_slot
    got = _same(pkg, ps)
    assert got["h"] == min(w.hx for w in ps)


def test_own_cell_partition(pkg):
    rng = np.random.default_rng(9)
    a = W.box(5, 5, 4, h=0.2, parts=(2, 2, 1), f='random', seed=3,
              holes=(((1, 3), (1, 3), (1, 2)),))
    a.cell_part = rng.integers(0, 5, a.nx * a.ny * a.nz).astype(np.int32)
    b = W.box(3, 2, 2, h=0.2, parts=(1, 1, 1), f='random', seed=4)
    got = _same(pkg, [a, b])
    act = got["cell_part"][got["active"] == 1]
    assert act.max() == 5  # five parts of a, then b's single box


def test_invalid_compositions_rejected(pkg):
    a = W.box(3, 3, 3, parts=(1, 1, 1))
    b = W.box(3, 3, 3, parts=(1, 1, 1), overlap=2)
    with pytest.raises(pkg.GeneoError) as e:
        pkg.compose([a, b])
    assert e.value.status == -1
    c = W.box(4, 2, 2, parts=(1, 1, 1))  # h = 1/4 in every direction, but
    c.hy = 0.3                           # non-cubic cells are refused
    with pytest.raises(pkg.GeneoError):
        pkg.compose([a, c])
    with pytest.raises(pkg.GeneoError):
        pkg.compose([])
