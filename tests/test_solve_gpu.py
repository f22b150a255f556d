"""The step after assembly on the GPU: y = K x on the assembled values and
the constrained equilibrium solve, against the oracle's CSR product and its
direct sparse solve."""
import numpy as np
import pytest
import torch

import oracle
from helpers import small_cases
from paper_2505_02438_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MAT = (1.0, 1e-9, 0.3, 3.0, 0)


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    return t if dtype is None else t.to(dtype)


@pytest.mark.parametrize("name,cell,k,coords,cells", small_cases(), ids=[c[0] for c in small_cases()])
def test_spmv_matches_oracle(lib, name, cell, k, coords, cells):
    m = lib.Mesh(cell, k, coords, cells, *MAT)
    g = np.random.default_rng(8)
    rho = g.uniform(0.001, 1.0, len(cells))
    vals = m.assemble_K(dev(rho))
    x = g.standard_normal(m.ndof)
    y = m.spmv(vals, dev(x)).cpu().numpy()
    rp, ci, v, ndof = oracle.assemble(cell, k, coords, cells, MAT, rho)
    want = oracle.spmv(rp, ci, v, x)
    scale = np.array([np.abs(v[rp[r]:rp[r + 1]]) @ np.abs(x[ci[rp[r]:rp[r + 1]]]) for r in range(ndof)])
    assert np.all(np.abs(y - want) <= 1e-12 * scale + 1e-300)
    assert torch.equal(m.spmv(vals, dev(x)), m.spmv(vals, dev(x)))


def cantilever(nx, ny, nz, jitter=0.0):
    """Hex box fixed on x = 0, a downward load spread over the nodes of x = nx."""
    coords, cells = W.hex_grid(nx, ny, nz, jitter, np.random.default_rng(3))
    return coords, cells


@pytest.mark.parametrize("check_every", [5, 10], ids=["launches", "graph"])
@pytest.mark.parametrize("cell,k,mk", [
    ("hex", 1, lambda: cantilever(12, 4, 4)),
    ("hex", 1, lambda: cantilever(10, 4, 3, jitter=0.15)),
    ("tet", 2, lambda: W.kuhn_tets(6, 2, 2, 0.15, np.random.default_rng(4))),
    ("quad", 2, lambda: W.quad_grid(12, 5, 0.2, np.random.default_rng(5))),
])
def test_cg_matches_direct_solve(lib, cell, k, mk, check_every):
    """Both loops: kernel by kernel (odd check interval) and replayed as a graph
    between checks (even interval)."""
    coords, cells = mk()
    m = lib.Mesh(cell, k, coords, cells, *MAT)
    d = m.dim
    rho = np.random.default_rng(6).uniform(0.3, 1.0, len(cells))
    vals = m.assemble_K(dev(rho))
    xn = oracle.node_coords(cell, k, coords, cells)
    L = xn[:, 0].max()
    fixed = np.repeat(xn[:, 0] < 1e-9, d)
    f = np.zeros(m.ndof)
    tip = np.where(xn[:, 0] > L - 1e-9)[0]
    f[d * tip + (d - 1)] = -1.0 / len(tip)
    u, info = m.solve(vals, dev(fixed), dev(f), rtol=1e-12, max_iter=20000, check_every=check_every)
    assert info["converged"] and info["rel_residual"] <= 1e-12
    rp, ci, v, ndof = oracle.assemble(cell, k, coords, cells, MAT, rho)
    ref = oracle.solve_dirichlet(rp, ci, v, fixed, f, np.zeros(ndof))
    un = u.cpu().numpy()
    assert np.linalg.norm(un - ref) <= 1e-8 * np.linalg.norm(ref)
    assert np.all(un[fixed] == 0.0)
    # same bits on a second solve
    u2, info2 = m.solve(vals, dev(fixed), dev(f), rtol=1e-12, max_iter=20000, check_every=check_every)
    assert torch.equal(u, u2) and info2["iterations"] == info["iterations"]


def test_cg_graph_replay_is_bitwise_the_launch_loop(lib):
    """A fixed number of iterations (the tolerance is never met) gives the same
    bits whether the iterations are replayed as a graph (check interval 10, also
    with a remainder of 7 launched one by one) or launched one by one (interval 3),
    and a new right-hand side reuses the kept graph with the new vectors."""
    coords, cells = cantilever(9, 3, 3)
    m = lib.Mesh("hex", 1, coords, cells, *MAT)
    rho = np.random.default_rng(7).uniform(0.3, 1.0, len(cells))
    vals = m.assemble_K(dev(rho))
    xn = oracle.node_coords("hex", 1, coords, cells)
    fixed = np.repeat(xn[:, 0] < 1e-9, 3)
    f = np.zeros(m.ndof)
    tip = np.where(xn[:, 0] > xn[:, 0].max() - 1e-9)[0]
    f[3 * tip + 2] = -1.0 / len(tip)
    for n in (40, 47):
        ug, ig = m.solve(vals, dev(fixed), dev(f), rtol=1e-300, max_iter=n, check_every=10)
        ul, il = m.solve(vals, dev(fixed), dev(f), rtol=1e-300, max_iter=n, check_every=3)
        assert ig["iterations"] == il["iterations"] == n
        assert torch.equal(ug, ul)
    f2 = 2.0 * f
    ug2, _ = m.solve(vals, dev(fixed), dev(f2), rtol=1e-300, max_iter=40, check_every=10)
    ul2, _ = m.solve(vals, dev(fixed), dev(f2), rtol=1e-300, max_iter=40, check_every=3)
    assert torch.equal(ug2, ul2)


def test_cg_patch_test_prescribed_affine_field(lib):
    """Homogeneous body, an affine displacement prescribed on the boundary, no
    load: the solve returns that field at every dof."""
    coords, cells = W.hex_grid(5, 4, 3, 0.15, np.random.default_rng(9))
    m = lib.Mesh("hex", 2, coords, cells, *MAT)
    vals = m.assemble_K(dev(np.full(len(cells), 0.6)))
    xn = oracle.node_coords("hex", 2, coords, cells)
    A = np.random.default_rng(1).standard_normal((3, 3))
    ulin = (xn @ A.T + 1.0).ravel()
    bnd = ~np.all((xn > 1e-9) & (xn < np.array([5, 4, 3]) - 1e-9), axis=1)
    fixed = np.repeat(bnd, 3)
    u, info = m.solve(vals, dev(fixed), dev(np.zeros(m.ndof)), u_fixed=dev(ulin), rtol=1e-13, max_iter=5000)
    assert info["converged"]
    assert np.abs(u.cpu().numpy() - ulin).max() <= 1e-9 * np.abs(ulin).max()


def test_cg_rejects_an_untouched_free_dof(lib):
    """A vertex no cell uses has an empty row: the Jacobi preconditioner is
    undefined there and the solve reports EINVAL instead of dividing by zero."""
    from paper_2505_02438_gb300 import _native as N
    coords, cells = W.structured_quad(3, 2)
    coords = np.vstack([coords, [[10.0, 10.0]]])
    m = lib.Mesh("quad", 1, coords, cells, *MAT)
    vals = m.assemble_K(dev(np.full(len(cells), 0.5)))
    fixed = np.zeros(m.ndof, bool)
    fixed[:2] = True
    with pytest.raises(N.SoptxError) as ei:
        m.solve(vals, dev(fixed), dev(np.ones(m.ndof)))
    assert ei.value.code == 1
