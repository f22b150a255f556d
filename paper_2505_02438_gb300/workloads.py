"""Seeded synthetic meshes and inputs for the SIMP assembly path.

This module only draws inputs: vertex coordinates, cell connectivity,
densities and displacements.  It holds none of the method's arithmetic (no
basis functions, element matrices, numbering of higher-order nodes or
assembly), so both the CUDA library and the CPU oracle can be fed from it.

Conventions of the generated meshes (grid spacing h = 1, as the paper's
``UniformMesh(..., h=[1, 1])`` examples use, Sec. 4):
  * vertices of an (nx+1) x (ny+1) [x (nz+1)] lattice, numbered
    lexicographically with x fastest;
  * quads / hexes: cells lexicographic (x fastest), corners in lexicographic
    order of the unit cell (x fastest);
  * triangles: every square split along its (i,j) -> (i+1,j+1) diagonal into
    (v00, v10, v11) and (v00, v11, v01), both counter-clockwise;
  * tetrahedra: every cube split into the 6 Kuhn (Freudenthal) tetrahedra
    along the (0,0,0) -> (1,1,1) diagonal, one per axis permutation, so the
    split is conforming across cubes;
  * jitter moves interior vertices only, each coordinate by U(-a h, a h), so
    the domain stays a box.

Seeds follow ``seed = 1000 * workload + stream`` with streams 0 = jitter,
1 = density, 2 = displacement, 3 = arrivals, 4 = mesh draws, using numpy's
PCG64 ``default_rng``.
"""
import itertools
from dataclasses import dataclass, field

import numpy as np

DIM = {"tri": 2, "tet": 3, "quad": 2, "hex": 3}
NVERT = {"tri": 3, "tet": 4, "quad": 4, "hex": 8}


def rng(workload, stream):
    return np.random.default_rng(1000 * int(workload) + int(stream))


def lattice_vertices(shape):
    """Vertices of a lattice with len(shape) axes of n cells each (x fastest)."""
    axes = [np.arange(n + 1, dtype=np.float64) for n in shape]
    grids = np.meshgrid(*axes, indexing="ij")
    # ij indexing gives x slowest; transpose so that x is fastest in memory
    pts = np.stack([g.transpose(tuple(range(len(shape)))[::-1]).ravel() for g in grids], axis=1)
    return pts


def _vid(shape, idx):
    """Lexicographic vertex id (x fastest) of lattice index tuples idx[..., d]."""
    vid = np.zeros(idx.shape[:-1], np.int64)
    stride = 1
    for m, n in enumerate(shape):
        vid += idx[..., m] * stride
        stride *= n + 1
    return vid


def _cell_origins(shape):
    axes = [np.arange(n) for n in shape]
    grids = np.meshgrid(*axes[::-1], indexing="ij")   # last axis slowest
    return np.stack([g.ravel() for g in grids[::-1]], axis=1)   # x fastest


def structured_quad(nx, ny):
    shape = (nx, ny)
    o = _cell_origins(shape)
    corners = np.array([[0, 0], [1, 0], [0, 1], [1, 1]])
    cells = _vid(shape, o[:, None, :] + corners[None])
    return lattice_vertices(shape), cells.astype(np.int32)


def structured_hex(nx, ny, nz):
    shape = (nx, ny, nz)
    o = _cell_origins(shape)
    corners = np.array([[i, j, l] for l in (0, 1) for j in (0, 1) for i in (0, 1)])
    cells = _vid(shape, o[:, None, :] + corners[None])
    return lattice_vertices(shape), cells.astype(np.int32)


def _jitter(coords, shape, amount, g):
    if amount == 0.0:
        return coords
    coords = coords.copy()
    n = len(coords)
    idx = np.zeros((n, len(shape)), np.int64)
    rem = np.arange(n)
    for m, s in enumerate(shape):
        idx[:, m] = rem % (s + 1)
        rem //= s + 1
    interior = np.all((idx > 0) & (idx < np.array(shape)), axis=1)
    shift = g.uniform(-amount, amount, size=coords.shape)
    coords[interior] += shift[interior]
    return coords


def quad_grid(nx, ny, jitter=0.0, g=None):
    """Quads of an nx x ny grid, interior vertices jittered (then the cells are
    general bilinear quadrilaterals, not parallelograms)."""
    coords, cells = structured_quad(nx, ny)
    return _jitter(coords, (nx, ny), jitter, g), cells


def hex_grid(nx, ny, nz, jitter=0.0, g=None):
    """Hexahedra of an nx x ny x nz grid, interior vertices jittered (general
    trilinear hexahedra)."""
    coords, cells = structured_hex(nx, ny, nz)
    return _jitter(coords, (nx, ny, nz), jitter, g), cells


def triangle_grid(nx, ny, jitter=0.0, g=None):
    shape = (nx, ny)
    o = _cell_origins(shape)
    v = lambda di, dj: _vid(shape, o + np.array([di, dj]))
    t1 = np.stack([v(0, 0), v(1, 0), v(1, 1)], axis=1)
    t2 = np.stack([v(0, 0), v(1, 1), v(0, 1)], axis=1)
    cells = np.stack([t1, t2], axis=1).reshape(-1, 3)
    coords = _jitter(lattice_vertices(shape), shape, jitter, g)
    return coords, cells.astype(np.int32)


def kuhn_tets(nx, ny, nz, jitter=0.0, g=None):
    shape = (nx, ny, nz)
    o = _cell_origins(shape)
    tets = []
    for perm in itertools.permutations(range(3)):
        path = [np.zeros(3, np.int64)]
        for ax in perm:
            step = path[-1].copy()
            step[ax] += 1
            path.append(step)
        tets.append(np.stack([_vid(shape, o + p) for p in path], axis=1))
    cells = np.stack(tets, axis=1).reshape(-1, 4)
    coords = _jitter(lattice_vertices(shape), shape, jitter, g)
    return coords, cells.astype(np.int32)


@dataclass
class Workload:
    """One synthetic assembly problem: mesh, order, material and inputs."""
    name: str
    cell: str
    order: int
    coords: np.ndarray
    cells: np.ndarray
    E0: float = 1.0
    Emin: float = 1e-9
    nu: float = 0.3
    p: float = 3.0
    plane_strain: int = 0
    rho: np.ndarray = None
    seed_base: int = 0
    elem_prec: str = "fp64"
    extra: dict = field(default_factory=dict)

    @property
    def dim(self):
        return DIM[self.cell]

    @property
    def mat(self):
        return (self.E0, self.Emin, self.nu, self.p, self.plane_strain)

    def displacement(self, ndof):
        """u ~ N(0, 1) per dof, seeded; ndof comes from the mesh numbering."""
        return rng(self.seed_base, 2).standard_normal(ndof)


def _rho_uniform(nc, g):
    return g.uniform(0.001, 1.0, size=nc)


def mbb_q4(nx=60, ny=20, wl=1):
    """Q4 plane stress on the MBB-beam rectangle; rho = 0.5 + U(-0.1, 0.1)."""
    coords, cells = structured_quad(nx, ny)
    rho = np.clip(0.5 + rng(wl, 1).uniform(-0.1, 0.1, size=len(cells)), 0.001, 1.0)
    return Workload("q4_%dx%d" % (nx, ny), "quad", 1, coords, cells, rho=rho, seed_base=wl)


def cantilever_hex(nx=120, ny=40, nz=40, order=1, wl=2):
    """Trilinear (or order-k) hex box, rho ~ U(0.001, 1)."""
    coords, cells = structured_hex(nx, ny, nz)
    rho = _rho_uniform(len(cells), rng(wl, 1))
    return Workload("hex_q%d_%dx%dx%d" % (order, nx, ny, nz), "hex", order, coords, cells,
                    rho=rho, seed_base=wl)


def jittered_tri(nx=400, ny=200, order=3, jitter=0.2, wl=3):
    """Triangles of an nx x ny grid, interior vertices jittered, plane stress."""
    coords, cells = triangle_grid(nx, ny, jitter, rng(wl, 0))
    rho = _rho_uniform(len(cells), rng(wl, 1))
    return Workload("tri_p%d_%dx%d" % (order, nx, ny), "tri", order, coords, cells,
                    rho=rho, seed_base=wl)


def jittered_tet(nx=60, ny=20, nz=20, order=2, jitter=0.15, wl=4):
    """Kuhn tetrahedra of an nx x ny x nz grid, interior vertices jittered."""
    coords, cells = kuhn_tets(nx, ny, nz, jitter, rng(wl, 0))
    rho = _rho_uniform(len(cells), rng(wl, 1))
    return Workload("tet_p%d_%dx%dx%d" % (order, nx, ny, nz), "tet", order, coords, cells,
                    rho=rho, seed_base=wl)


def jittered_quad(nx=60, ny=20, order=1, jitter=0.2, wl=6):
    """Bilinear quadrilaterals (interior vertices jittered), plane stress."""
    coords, cells = quad_grid(nx, ny, jitter, rng(wl, 0))
    rho = _rho_uniform(len(cells), rng(wl, 1))
    return Workload("quadj_q%d_%dx%d" % (order, nx, ny), "quad", order, coords, cells, rho=rho, seed_base=wl)


def jittered_hex(nx=120, ny=40, nz=40, order=1, jitter=0.15, wl=7):
    """Trilinear hexahedra of the cantilever box, interior vertices jittered."""
    coords, cells = hex_grid(nx, ny, nz, jitter, rng(wl, 0))
    rho = _rho_uniform(len(cells), rng(wl, 1))
    return Workload("hexj_q%d_%dx%dx%d" % (order, nx, ny, nz), "hex", order, coords, cells, rho=rho, seed_base=wl)


def standard(i, scale=1.0):
    """The five standard workloads at full size (scale=1) or shrunk per axis."""
    s = lambda n: max(1, int(round(n * scale)))
    if i == 1:
        return mbb_q4(s(60), s(20))
    if i == 2:
        return cantilever_hex(s(120), s(40), s(40))
    if i == 3:
        return jittered_tri(s(400), s(200))
    if i == 4:
        return jittered_tet(s(60), s(20), s(20))
    raise ValueError("workload %r has no single mesh" % i)


def serving_stream(n_jobs=64, iters=8, wl=5, scale=1.0):
    """The serving workload: n_jobs design jobs x iters requests.  Each job is a
    mesh family drawn uniformly from {Q4 plane stress, hex Q1, Kuhn P2 tets}
    with a size from t ~ U(0, 1) (Q4 from 60x20 to 800x400, hex from 30x10x10
    to 120x40x40, tet cubes from 6x2x2 to 60x20x20, each axis shrunk by
    `scale`), and FP64 or FP32 element matrices with probability 1/2.
    Returns a list of jobs: dict(job, workload, elem_prec)."""
    g = rng(wl, 4)
    jobs = []
    for j in range(n_jobs):
        fam = int(g.integers(0, 3))
        t = float(g.uniform(0.0, 1.0))
        prec = "fp64" if g.uniform() < 0.5 else "fp32"
        s = lambda n: max(1, int(round(n * scale)))
        if fam == 0:
            w = mbb_q4(s(60 * (800 / 60) ** t), s(20 * (400 / 20) ** t), wl=100 + j)
        elif fam == 1:
            f = 4 ** t
            w = cantilever_hex(s(30 * f), s(10 * f), s(10 * f), wl=100 + j)
        else:
            f = 10 ** t
            w = jittered_tet(s(6 * f), s(2 * f), s(2 * f), wl=100 + j)
        w.elem_prec = prec
        jobs.append(dict(job=j, workload=w, elem_prec=prec))
    return jobs


def small_serving_stream(n_jobs=256, wl=6):
    """Many small design jobs: Q4 plane-stress boxes with log-uniform sides
    from 16 x 16 to 64 x 64 cells (the sizes the grouped step serves), FP64.
    Returns a list of jobs: dict(job, workload, elem_prec)."""
    g = rng(wl, 4)
    jobs = []
    for j in range(n_jobs):
        nx = int(round(16 * 4 ** float(g.uniform(0.0, 1.0))))
        ny = int(round(16 * 4 ** float(g.uniform(0.0, 1.0))))
        w = mbb_q4(nx, ny, wl=200 + j)
        w.elem_prec = "fp64"
        jobs.append(dict(job=j, workload=w, elem_prec="fp64"))
    return jobs


def poisson_arrivals(n, rate_per_s, wl=5):
    """Arrival times (seconds) of n requests at the given Poisson rate."""
    return np.cumsum(rng(wl, 3).exponential(1.0 / rate_per_s, size=n))


def cantilever_3d_oc(nx=60, ny=20, nz=4):
    """The 3D cantilever of the paper's Sec. 5.4: a box of nx x ny x nz unit
    hexahedra, the x = 0 face fixed, a downward load (-1 along y) on every node
    of the bottom edge of the right end (x = nx, y = 0).  Returns
    (workload, fixed dof mask [ndof] bool, load [ndof]) with dofs
    node-interleaved and the vertex lattice as the node numbering."""
    coords, cells = structured_hex(nx, ny, nz)
    wl = Workload("cantilever3d_%dx%dx%d" % (nx, ny, nz), "hex", 1, coords, cells, rho=np.full(len(cells), 0.3),
                  seed_base=8)
    ndof = 3 * len(coords)
    fixed = np.repeat(coords[:, 0] < 1e-9, 3)
    f = np.zeros(ndof)
    tip = np.nonzero((coords[:, 0] > nx - 1e-9) & (coords[:, 1] < 1e-9))[0]
    f[3 * tip + 1] = -1.0
    return wl, fixed, f
