"""Integer set-up data of the library against the oracle, bit for bit, on
the CPU: geneo_setup_topology runs the host part of the set-up without any
CUDA call.  Mesh edges, Dirichlet flags, unknown numbering, CSR pattern,
subdomain index sets N_i, partition-of-unity owners, split near-kernel
columns and k0/k1 must be identical to the oracle's (oracle/mesh.py,
oracle/dd.py, oracle/coarse.py) on the parity cases, the 32^3 benchmark
workload, an explicit cell partition, composed independent problems and
natural (Neumann) boundary faces on lateral sides and hole surfaces;
the kept vertices of every local gradient G_j as well; compute calls on
such a context are refused with STATE."""
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


def _hetero(seed=0, parts=(3, 2, 1), overlap=1, n=(10, 8, 6), holes=(((4, 6), (3, 5), (0, 6)),)):
    rng = np.random.default_rng(seed)
    nc = n[0] * n[1] * n[2]
    return W.box(*n, parts=parts, overlap=overlap, gamma=1e-3,
                 mu_inv=10.0 ** rng.uniform(0, 2, nc), eps=10.0 ** rng.uniform(-0.5, 0.5, nc),
                 holes=holes, f='random', seed=seed, tau=0.1)


def _composite():
    rng = np.random.default_rng(5)
    a = W.box(6, 6, 6, h=1 / 6, parts=(2, 1, 1), gamma=1e-2, mu_inv=10.0 ** rng.uniform(0, 2, 216),
              f='random', seed=1, holes=(((2, 4), (2, 4), (1, 5)),))
    b = W.box(5, 4, 4, h=1 / 6, parts=(1, 2, 1), f='random', seed=2)
    return W.compose([a, b])


def _metis_like():
    w = _hetero(seed=3, parts=(1, 1, 1), holes=())
    rng = np.random.default_rng(4)
    # an irregular partition: random seeds grown by distance (Voronoi cells)
    c = np.arange(w.nx * w.ny * w.nz)
    xyz = np.stack([c % w.nx, (c // w.nx) % w.ny, c // (w.nx * w.ny)], 1)
    seeds = xyz[rng.choice(len(c), 7, replace=False)]
    w.cell_part = np.argmin(((xyz[:, None, :] - seeds[None]) ** 2).sum(-1), 1).astype(np.int32)
    return w


def _natural(w, **kw):
    w.natural = W.natural_faces(w, **kw)
    return w


CASES = {
    "cube8": W.unit_cube_8,
    "hetero_hole": lambda: _hetero(),
    "overlap2": lambda: _hetero(seed=1, parts=(2, 2, 1), overlap=2, n=(9, 9, 5), holes=()),
    "one_sub": lambda: _hetero(seed=2, parts=(1, 1, 1), n=(5, 4, 4), holes=()),
    "ragged_beam": lambda: W.box(13, 3, 3, h=1 / 3, parts=(4, 1, 1), overlap=1, gamma=0.5),
    "cube32_hole_channels": W.cube32_hole_channels,
    "voronoi_partition": _metis_like,
    "composite": _composite,
    # a batching cube with a box whose edges all join boundary vertices
    # (no kept vertex, an empty G_j)
    "batch35_n9": lambda: [w for w in W.many_problems(256, seed=3) if w.nx <= 10][4],
    # natural (Neumann) boundary faces, Sec. 4's mixed conditions
    "beam_mixed": lambda: _natural(W.box(16, 4, 4, h=0.25, parts=(4, 1, 1)),
                                   sides=((1, 0), (1, 1))),
    "holes_natural": lambda: _natural(_hetero(seed=5), holes=True),
    "beam_holes_natural": lambda: W.beam_holes(4),
    "beam_holes_dirichlet": lambda: W.beam_holes(4, natural_holes=False),
    "all_natural": lambda: _natural(W.box(5, 4, 3, parts=(2, 2, 1), holes=(((2, 3), (1, 3), (1, 2)),)),
                                    holes=True, sides=[(a, s) for a in range(3) for s in (0, 1)]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_integer_setup_matches_oracle(pkg, name):
    from oracle.mesh import build_mesh
    from oracle.fem import assemble_A
    from oracle.dd import decompose, k0, k1
    from oracle.coarse import snk_columns
    w = CASES[name]()
    s = pkg.Solver.topology(w)
    m = build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active,
                   natural=getattr(w, "natural", None))
    dec = decompose(m, w.parts, w.overlap, cell_part=getattr(w, "cell_part", None))
    assert np.array_equal(s.export("edges").reshape(-1, 2), m.edges)
    assert np.array_equal(s.export("dir_edge").astype(bool), m.dir_edge)
    assert np.array_equal(s.export("dof_edge"), m.dof_edge)
    assert np.array_equal(s.export("dof_vert"), m.dof_vert)
    A = assemble_A(m, w)
    assert np.array_equal(s.export("A_rowptr"), A.indptr)
    assert np.array_equal(s.export("A_col"), A.indices)
    noff, nidx = s.export("N_off"), s.export("N_idx")
    assert len(noff) == dec.nsub + 1 == s.sizes["nsub"] + 1
    for i in range(dec.nsub):
        assert np.array_equal(nidx[noff[i]:noff[i + 1]], dec.N[i])
    assert np.array_equal(s.export("owner"), dec.owner)
    snk = snk_columns(m, dec)
    assert np.array_equal(s.export("snk_sub"), np.array([c[0] for c in snk], np.int32))
    assert np.array_equal(s.export("snk_vert"), np.array([c[1] for c in snk], np.int32))
    assert s.sizes["n0_snk"] == len(snk)
    zp, zr, zv = s.export("Zcol_ptr"), s.export("Zcol_row"), s.export("Zcol_val")
    assert len(zp) == len(snk) + 1
    for k, (_, _, rows, vals) in enumerate(snk):
        assert np.array_equal(zr[zp[k]:zp[k + 1]], rows)
        assert np.array_equal(zv[zp[k]:zp[k + 1]], vals)
    assert list(s.export("k0k1")) == [k0(A, dec), k1(dec)]
    from oracle.coarse import local_gradient
    xo, xv = s.export("xv_off"), s.export("xv_vert")
    for j in range(dec.nsub):
        assert np.array_equal(xv[xo[j]:xo[j + 1]], local_gradient(m, dec, j)[1])
    s.close()


def test_composite_components(pkg):
    """Composed problems: one contiguous unknown range per problem, in
    problem order, each the size of the problem alone."""
    from oracle.mesh import build_mesh
    rng = np.random.default_rng(5)
    ps = [W.box(6, 6, 6, h=1 / 6, parts=(2, 1, 1), gamma=1e-2,
                mu_inv=10.0 ** rng.uniform(0, 2, 216)),
          W.box(5, 4, 4, h=1 / 6, parts=(1, 2, 1)),
          W.box(4, 4, 3, h=1 / 6, parts=(2, 1, 1))]
    s = pkg.Solver.topology(W.compose(ps))
    off = s.export("seg_off")
    sizes = [build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active).ndofs for w in ps]
    assert list(np.diff(off)) == sizes
    s.close()


def test_compute_calls_refused(pkg):
    s = pkg.Solver.topology(W.unit_cube_8())
    for name in ("A_val", "loc_f32"):
        with pytest.raises(pkg.GeneoError) as e:
            s.export(name)
        assert e.value.status == -7
    lib = pkg.load_library()
    assert lib.geneo_use_precision(s._ctx, pkg.PREC_FP64) == -7
    assert lib.geneo_solve(s._ctx, None, None, 1e-8, 10, None, None) == -7
    s.close()


@pytest.mark.parametrize("name", ["hetero_hole", "beam_holes_natural", "cube8", "all_natural"])
def test_global_near_kernel_columns(pkg, name):
    """coarse = NK (Sec. 4, AS-NK): one gradient column per interior vertex,
    minus the highest vertex of each component with no Dirichlet vertex,
    equal to the oracle's nk_columns (rows and signs).  On the all-natural
    box (one floating component) exactly one column is dropped, and the kept
    columns have full rank: the incidence matrix of a connected graph has
    rank (vertices - 1), so G minus any one column is injective."""
    from oracle.mesh import build_mesh
    from oracle.coarse import nk_columns, assemble_Z
    w = CASES[name]()
    s = pkg.Solver.topology(w, coarse=pkg.COARSE_NK)
    m = build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active,
                   natural=getattr(w, "natural", None))
    ref = nk_columns(m)
    floating = 1 if name == "all_natural" else 0
    assert s.sizes["n0_snk"] == len(ref) == m.nvdofs - floating
    if floating:
        Z = assemble_Z(m.ndofs, ref).toarray()
        assert np.linalg.matrix_rank(Z) == Z.shape[1]
        assert ref[-1][1] < m.dof_vert.max()  # the highest vertex is the one dropped
    zp, zr, zv = s.export("Zcol_ptr"), s.export("Zcol_row"), s.export("Zcol_val")
    assert np.array_equal(s.export("snk_vert"), np.array([c[1] for c in ref], np.int32))
    for k, (_, _, rows, vals) in enumerate(ref):
        o = np.argsort(rows)
        assert np.array_equal(zr[zp[k]:zp[k + 1]], rows[o])
        assert np.array_equal(zv[zp[k]:zp[k + 1]], vals[o])
    s.close()


def test_invalid_problems_rejected_without_gpu(pkg):
    """Argument checks of the set-up (shared by geneo_setup and
    geneo_setup_topology) on the CPU: each bad input gives INVALID_ARG (-1)
    and no context."""
    def expect_invalid(w, **opt):
        with pytest.raises(pkg.GeneoError) as e:
            pkg.Solver.topology(w, **opt)
        assert e.value.status == -1
    ok = W.box(4, 3, 3, parts=(2, 1, 1))
    s = pkg.Solver.topology(ok)
    assert s.sizes["nsub"] == 2
    s.close()
    bad = W.box(4, 3, 3, parts=(2, 1, 1), gamma=1.0)
    bad.gamma = 0.0
    expect_invalid(bad)
    bad = W.box(4, 3, 3, parts=(2, 1, 1))
    bad.overlap = 0
    expect_invalid(bad)
    bad = W.box(4, 3, 3, parts=(5, 1, 1))
    expect_invalid(bad)
    bad = W.box(4, 3, 3, parts=(2, 1, 1))
    bad.mu_inv = np.where(np.arange(36) == 7, -1.0, 1.0)
    expect_invalid(bad)
    bad = W.box(4, 3, 3, parts=(2, 1, 1))
    bad.cell_part = np.full(36, -2, np.int32)
    expect_invalid(bad)
    # no active cell: no unknown at all
    expect_invalid(W.box(2, 2, 2, parts=(1, 1, 1), holes=(((0, 2), (0, 2), (0, 2)),)))
    # one cell still has one unknown, its body diagonal (the only edge off the faces)
    one = pkg.Solver.topology(W.box(1, 1, 1, parts=(1, 1, 1)))
    assert one.n == 1
    one.close()
    expect_invalid(ok, lobpcg_block=17)
    expect_invalid(ok, coarse=3)
    expect_invalid(ok, lobpcg_neumann=2)
