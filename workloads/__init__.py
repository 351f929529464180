"""Seeded synthetic inputs for the positive-Maxwell GenEO workloads.

This module only draws inputs: grid shape, active-cell masks (holes), per-cell
coefficients mu^-1 and eps, gamma, the box partition, the overlap width, the
GenEO threshold and the source field.  It holds none of the method's
arithmetic, so the CPU oracle and the CUDA library both consume it.

Conventions (the library's C-ABI uses the same ones):

* cells are numbered ``c = i + nx*(j + ny*k)``;
* vertices are numbered ``v = i + (nx+1)*(j + (ny+1)*k)``;
* the source field is given per *edge slot* ``(v, d)``: every edge of the
  Kuhn-split structured mesh runs from its lower vertex ``v`` along one of the
  seven positive directions ``DIRS[d]``.  ``f_slot`` has shape
  ``[nrhs, nverts, 7, 3]`` (float64); slots that are not edges are ignored.

The workloads follow the paper's test set-up (cubic cells split into six
tetrahedra, beams of size (N/2)x1x1 with h=1/16, layered or hole-located
coefficient jumps, gamma between 1e-6 and 1e2; Section 4) and the five
configurations this library is benchmarked on.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

# positive edge directions of the Kuhn split (axis, face diagonal, body diagonal)
DIRS = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1],
                 [1, 1, 0], [1, 0, 1], [0, 1, 1], [1, 1, 1]], dtype=np.int64)


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float
    active: np.ndarray          # uint8 [ncells]
    mu_inv: np.ndarray          # float64 [ncells]
    eps: np.ndarray             # float64 [ncells]
    gamma: float
    parts: tuple                # (px, py, pz) boxes
    overlap: int                # layers of cells added around each box
    tau: float                  # GenEO threshold (convention chosen by the solver)
    f_slot: np.ndarray          # float64 [nrhs, nverts, 7, 3]
    meta: dict = field(default_factory=dict)
    cell_part: np.ndarray = None  # int32 [ncells] explicit subdomain per cell, or None (boxes)
    natural: np.ndarray = None    # uint8 [ncells] natural boundary faces (bit 2a + side), or None

    @property
    def ncells(self):
        return self.nx * self.ny * self.nz

    @property
    def nverts(self):
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def nrhs(self):
        return self.f_slot.shape[0]


def _cell_ijk(nx, ny, nz):
    c = np.arange(nx * ny * nz)
    return c % nx, (c // nx) % ny, c // (nx * ny)


def _const_f(nverts, vec=(1.0, 1.0, 1.0), nrhs=1):
    f = np.empty((nrhs, nverts, 7, 3), dtype=np.float64)
    f[...] = np.asarray(vec, dtype=np.float64)
    return f


def _uniform_f(rng, nverts, nrhs=1):
    return rng.uniform(-1.0, 1.0, size=(nrhs, nverts, 7, 3))


def box(nx, ny, nz, *, h=None, parts=(2, 2, 2), overlap=1, gamma=1.0, tau=0.1,
        mu_inv=1.0, eps=1.0, holes=(), f=(1.0, 1.0, 1.0), nrhs=1, seed=None,
        name=None):
    """Generic box of cells.  ``holes`` lists half-open cell ranges
    ``((i0,i1),(j0,j1),(k0,k1))`` that are removed.  ``mu_inv``/``eps`` are
    scalars or per-cell arrays.  ``f`` is a constant 3-vector or ``'random'``
    (uniform in [-1,1]^3 per edge slot, seeded)."""
    if h is None:
        h = 1.0 / max(nx, ny, nz)
    ncells = nx * ny * nz
    ci, cj, ck = _cell_ijk(nx, ny, nz)
    active = np.ones(ncells, dtype=np.uint8)
    for (i0, i1), (j0, j1), (k0, k1) in holes:
        m = (ci >= i0) & (ci < i1) & (cj >= j0) & (cj < j1) & (ck >= k0) & (ck < k1)
        active[m] = 0
    mu = np.broadcast_to(np.asarray(mu_inv, dtype=np.float64), (ncells,)).copy()
    ep = np.broadcast_to(np.asarray(eps, dtype=np.float64), (ncells,)).copy()
    nverts = (nx + 1) * (ny + 1) * (nz + 1)
    if isinstance(f, str) and f == 'random':
        fs = _uniform_f(np.random.default_rng(seed), nverts, nrhs)
    else:
        fs = _const_f(nverts, f, nrhs)
    return Workload(name or f"box{nx}x{ny}x{nz}", nx, ny, nz, h, h, h, active, mu, ep,
                    float(gamma), tuple(parts), int(overlap), float(tau), fs)


def unit_cube_8():
    """Plain method, FP64: 8^3 unit cube, mu=eps=1, gamma=1, f=(1,1,1),
    2x2x2 boxes, one overlap layer, tau=0.1."""
    return box(8, 8, 8, parts=(2, 2, 2), overlap=1, gamma=1.0, tau=0.1,
               name="cube8_plain")


def cube32_hole_channels(seed=2):
    """32^3 unit cube with a through-hole (central 8x8x32 column removed);
    mu^-1 log-uniform in [1,1e3] per cell inside 4 random 2x2-cell channels
    running the full length of a random axis, 1 elsewhere; eps=1;
    gamma=1e-4; f uniform in [-1,1]^3 per edge; 4x4x4 boxes, overlap 2."""
    n = 32
    rng = np.random.default_rng(seed)
    ci, cj, ck = _cell_ijk(n, n, n)
    ijk = np.stack([ci, cj, ck])
    active = np.ones(n ** 3, dtype=np.uint8)
    active[(ci >= 12) & (ci < 20) & (cj >= 12) & (cj < 20)] = 0
    mu = np.ones(n ** 3)
    chans = []
    for _ in range(4):
        axis = int(rng.integers(0, 3))
        others = [a for a in range(3) if a != axis]
        p = int(rng.integers(0, n - 1))
        q = int(rng.integers(0, n - 1))
        m = ((ijk[others[0]] >= p) & (ijk[others[0]] < p + 2) &
             (ijk[others[1]] >= q) & (ijk[others[1]] < q + 2))
        mu[m] = 10.0 ** rng.uniform(0.0, 3.0, size=int(m.sum()))
        chans.append((axis, p, q))
    f = _uniform_f(rng, (n + 1) ** 3, 1)
    w = Workload("cube32_hole_channels", n, n, n, 1.0 / n, 1.0 / n, 1.0 / n, active, mu,
                 np.ones(n ** 3), 1e-4, (4, 4, 4), 2, 0.1, f, meta={"channels": chans})
    return w


def cube16_hole_channels(seed=2):
    """Profiling-size companion of cube32_hole_channels: 16^3 unit cube with
    a through-hole (central 4x4x16 column removed); mu^-1 log-uniform in
    [1,1e3] per cell inside 4 random 1x1-cell channels along a random axis,
    1 elsewhere; eps=1; gamma=1e-4; f uniform in [-1,1]^3 per edge;
    4x4x4 boxes, overlap 1 (local factors ~0.3 GB in float32)."""
    n = 16
    rng = np.random.default_rng(seed)
    ci, cj, ck = _cell_ijk(n, n, n)
    ijk = np.stack([ci, cj, ck])
    active = np.ones(n ** 3, dtype=np.uint8)
    active[(ci >= 6) & (ci < 10) & (cj >= 6) & (cj < 10)] = 0
    mu = np.ones(n ** 3)
    for _ in range(4):
        axis = int(rng.integers(0, 3))
        others = [a for a in range(3) if a != axis]
        p = int(rng.integers(0, n))
        q = int(rng.integers(0, n))
        m = (ijk[others[0]] == p) & (ijk[others[1]] == q)
        mu[m] = 10.0 ** rng.uniform(0.0, 3.0, size=int(m.sum()))
    f = _uniform_f(rng, (n + 1) ** 3, 1)
    return Workload("cube16_hole_channels", n, n, n, 1.0 / n, 1.0 / n, 1.0 / n, active, mu,
                    np.ones(n ** 3), 1e-4, (4, 4, 4), 1, 0.1, f)


def beam128_layered(seed=4, nrhs=16, nx=128, name="beam128_layered", gamma=1e-6,
                    contrast=1e6):
    """128x16x16 cells (h=1/16), two 4x4-cell through-holes along x
    (y in [3,7) and [9,13), z in [6,10)); mu^-1 alternating 1 and 1e6 every
    8 cells in x; eps=1; gamma=1e-6; 16 seeded uniform right-hand sides;
    32x4x4 boxes (one box per 4 cells along x), overlap 1."""
    ny, nz = 16, 16
    rng = np.random.default_rng(seed)
    ci, cj, ck = _cell_ijk(nx, ny, nz)
    active = np.ones(nx * ny * nz, dtype=np.uint8)
    for j0, j1 in ((3, 7), (9, 13)):
        active[(cj >= j0) & (cj < j1) & (ck >= 6) & (ck < 10)] = 0
    mu = np.where((ci // 8) % 2 == 0, 1.0, contrast)
    f = _uniform_f(rng, (nx + 1) * (ny + 1) * (nz + 1), nrhs)
    return Workload(name, nx, ny, nz, 1 / 16, 1 / 16, 1 / 16, active, mu,
                    np.ones(nx * ny * nz), gamma, (nx // 4, 4, 4), 1, 0.1, f)


def beam128_mild(seed=4, nrhs=16):
    """beam128_layered with gamma = 1e-3 and a 1e3 jump of mu^-1, where the
    float32 and bfloat16 split local factors stay definite."""
    return beam128_layered(seed, nrhs, name="beam128_mild", gamma=1e-3, contrast=1e3)


def beam64_layered(seed=4, nrhs=16):
    """Profiling-size companion of beam128_layered: the same beam cut to
    64 cells along x (16x4x4 boxes)."""
    return beam128_layered(seed, nrhs, nx=64, name="beam64_layered")


def cube48_blocks(seed=5, n=48, parts=8, name="cube48_blocks"):
    """48^3 unit cube, mu^-1 log-uniform in [1,1e6] on 3x3x3-cell blocks,
    gamma=1e-3, 8x8x8 boxes, overlap 1, f=(1,1,1)."""
    rng = np.random.default_rng(seed)
    ci, cj, ck = _cell_ijk(n, n, n)
    nb = (n + 2) // 3
    blk = 10.0 ** rng.uniform(0.0, 6.0, size=(nb, nb, nb))
    mu = blk[ck // 3, cj // 3, ci // 3]
    return Workload(name, n, n, n, 1 / n, 1 / n, 1 / n,
                    np.ones(n ** 3, dtype=np.uint8), mu, np.ones(n ** 3), 1e-3,
                    (parts, parts, parts), 1, 0.1, _const_f((n + 1) ** 3))


def cube24_blocks(seed=5):
    """cube48_blocks at 24^3 with 4x4x4 boxes (same subdomain size, 64
    subdomains)."""
    return cube48_blocks(seed, n=24, parts=4, name="cube24_blocks")


def paper_beam(nsub=8, *, gamma=1e-3, tau=0.1):
    """The paper's weak-scaling beam (N/2)x1x1 with h=1/16 and N boxes along
    the length, one overlap layer, mu=eps=1, f=(1,1,1) (Section 4)."""
    nx = 8 * nsub
    return box(nx, 16, 16, h=1 / 16, parts=(nsub, 1, 1), overlap=1, gamma=gamma,
               tau=tau, name=f"paper_beam_N{nsub}")


def many_problems(count=256, seed=3):
    """Batch of independent problems: n^3 cubes, n uniform in {8..24}, 1-2
    cubic holes of side U{2..ceil(n/4)} at least one cell from the boundary,
    mu^-1 in {1,1e2,1e4} on 4^3-cell blocks, gamma log-uniform in [1e-6,1],
    boxes (px,py,pz) in {2,3,4}^3 with product in [8,64], overlap 1."""
    rng = np.random.default_rng(seed)
    out = []
    choices = [(a, b, c) for a in (2, 3, 4) for b in (2, 3, 4) for c in (2, 3, 4)
               if 8 <= a * b * c <= 64]
    for p in range(count):
        n = int(rng.integers(8, 25))
        holes = []
        for _ in range(int(rng.integers(1, 3))):
            s = int(rng.integers(2, -(-n // 4) + 1))
            lo = [int(rng.integers(1, n - s)) for _ in range(3)]
            holes.append(tuple((l, l + s) for l in lo))
        ci, cj, ck = _cell_ijk(n, n, n)
        nb = -(-n // 4)
        blk = rng.choice(np.array([1.0, 1e2, 1e4]), size=(nb, nb, nb))
        mu = blk[ck // 4, cj // 4, ci // 4]
        gamma = float(10.0 ** rng.uniform(-6.0, 0.0))
        parts = choices[int(rng.integers(0, len(choices)))]
        w = box(n, n, n, parts=parts, overlap=1, gamma=gamma, tau=0.1, mu_inv=mu,
                holes=holes, name=f"batch{p}_n{n}")
        out.append(w)
    return out


def compose(problems, name="composite"):
    """Independent problems in one grid: problem p is placed at z offset
    zoff[p] (one inactive cell layer between consecutive problems) and at
    x = y = 0, cells outside it inactive.  gamma_p is folded into eps
    (the composite has gamma = 1), each problem keeps its own boxes through
    an explicit cell partition (its boxes, or its own cell_part offset past
    the previous problems' parts), and its edge-slot source field is copied
    to its vertices.  Cubic cells of another size h_p are mapped onto the
    composite's size H (the smallest) exactly: with lowest-order edge
    elements the curl-curl term of a tetrahedron scales as 1/h, the mass
    term as h and the load as h^2, so with r = h_p / H the same matrix and
    right-hand side come from mu^-1 / r, gamma eps r and f r^2.  All problems
    must share the overlap and tau.  meta["zoff"] records the offsets."""
    for w in problems:
        assert w.natural is None, "natural boundary faces are not supported here"
        assert w.hx == w.hy == w.hz and w.overlap == problems[0].overlap
        assert w.tau == problems[0].tau and w.nrhs == problems[0].nrhs
    h = min(w.hx for w in problems)
    nx = max(w.nx for w in problems)
    ny = max(w.ny for w in problems)
    zoff, z = [], 0
    for w in problems:
        zoff.append(z)
        z += w.nz + 1
    nz = z - 1
    nc = nx * ny * nz
    active = np.zeros(nc, dtype=np.uint8)
    mu = np.ones(nc)
    eps = np.ones(nc)
    part = np.zeros(nc, dtype=np.int32)
    nv = (nx + 1) * (ny + 1) * (nz + 1)
    f = np.zeros((problems[0].nrhs, nv, 7, 3))
    pbase = 0
    for w, zo in zip(problems, zoff):
        ci, cj, ck = _cell_ijk(w.nx, w.ny, w.nz)
        g = ci + nx * (cj + ny * (ck + zo))
        r = w.hx / h
        active[g] = w.active
        mu[g] = np.asarray(w.mu_inv, dtype=np.float64) / r
        eps[g] = np.asarray(w.eps, dtype=np.float64) * w.gamma * r
        if w.cell_part is not None:
            own = np.where(w.active == 1, np.asarray(w.cell_part, dtype=np.int64), 0)
            part[g] = pbase + own
            pbase += int(own[w.active == 1].max()) + 1
        else:
            px, py, pz = w.parts
            part[g] = pbase + (ci * px // w.nx) + px * ((cj * py // w.ny) + py * (ck * pz // w.nz))
            pbase += px * py * pz
        v = np.arange(w.nverts)
        vi = v % (w.nx + 1)
        vj = (v // (w.nx + 1)) % (w.ny + 1)
        vk = v // ((w.nx + 1) * (w.ny + 1))
        f[:, vi + (nx + 1) * (vj + (ny + 1) * (vk + zo))] = w.f_slot * (r * r)
    return Workload(name, nx, ny, nz, h, h, h, active, mu, eps, 1.0, (1, 1, 1),
                    problems[0].overlap, problems[0].tau, f, meta={"zoff": zoff},
                    cell_part=part)


def natural_faces(w, holes=False, sides=()):
    """Natural (Neumann) boundary faces of workload w as a uint8 mask per
    cell, bit 2a + s for the face on axis a (0, 1, 2 = x, y, z) at the lower
    (s = 0) or upper (s = 1) side of the cell.  holes=True marks every face
    towards an inactive cell inside the grid (the hole surfaces of Sec. 4);
    sides lists (a, s) pairs of the grid's outer faces to mark (e.g. two
    opposite lateral faces of the beam: ((1, 0), (1, 1))).  Other boundary
    faces stay Dirichlet."""
    nx, ny, nz = w.nx, w.ny, w.nz
    act = np.asarray(w.active).reshape(nz, ny, nx).astype(bool)
    mask = np.zeros((nz, ny, nx), dtype=np.uint8)
    n = (nx, ny, nz)
    for a in range(3):
        ax = 2 - a  # array axis of grid axis a (k, j, i order)
        for s in (0, 1):
            if holes:
                nb = np.zeros_like(act)
                src = [slice(None)] * 3
                dst = [slice(None)] * 3
                if s == 0:
                    src[ax], dst[ax] = slice(0, n[a] - 1), slice(1, n[a])
                else:
                    src[ax], dst[ax] = slice(1, n[a]), slice(0, n[a] - 1)
                nb[tuple(dst)] = ~act[tuple(src)]  # neighbour inside the grid and inactive
                mask |= (nb & act).astype(np.uint8) << (2 * a + s)
            if (a, s) in tuple(sides):
                edge = [slice(None)] * 3
                edge[ax] = 0 if s == 0 else n[a] - 1
                layer = np.zeros_like(act)
                layer[tuple(edge)] = True
                mask |= (layer & act).astype(np.uint8) << (2 * a + s)
    return mask.reshape(-1)


def beam_holes(nsub=4, m=8, natural_holes=True, gamma=1e-3, tau=0.1):
    """The beam with holes of Sec. 4 at mesh size h = 1/m: (nsub/2) x 1 x 1,
    nsub boxes along x, overlap 1.  Four square holes (side h * max(1, m/8))
    run along the whole length at y, z in {m/4, 3m/4 - 1} cells; in every
    box two square holes cross from the lateral face y = 0 to y = 1, at
    z = m/4 (a quarter into the box) and at z = 3m/4 - 1 (three quarters
    in), each meeting two of the length holes.  The hole sizes and
    positions are a reading of the paper's description (its figure is not
    available).  natural_holes: Neumann conditions on the hole surfaces
    (Sec. 4, mixed), the outer faces Dirichlet; else Dirichlet everywhere."""
    nx, ny, nz = nsub * m // 2, m, m
    L = nx // nsub
    a, b = m // 4, m - m // 4 - 1
    s = max(1, m // 8)
    holes = [((0, nx), (y, y + s), (z, z + s)) for (y, z) in ((a, a), (a, b), (b, a), (b, b))]
    for q in range(nsub):
        x0 = q * L
        holes.append(((x0 + L // 4, x0 + L // 4 + s), (0, ny), (a, a + s)))
        holes.append(((x0 + 3 * L // 4 - s, x0 + 3 * L // 4), (0, ny), (b, b + s)))
    w = box(nx, ny, nz, h=1.0 / m, parts=(nsub, 1, 1), overlap=1, gamma=gamma, tau=tau,
            holes=holes, name=f"beam_holes_{nsub}_{'natural' if natural_holes else 'dirichlet'}")
    if natural_holes:
        w.natural = natural_faces(w, holes=True)
    return w
