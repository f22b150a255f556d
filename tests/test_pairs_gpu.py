"""The pair kernel of 2D meshes (k_contract_pairs: the contraction of FP32
element matrices, and the reading of cached FP64 ones) at its edges: a
triangle fan whose centre meets 150 cells (a pair with more cells than a chunk
stages in shared memory, so its records past those come from global memory),
every order 1-3, both element precisions; moduli outside the float-pair range
on that fan (the lane's FP64 redo); repeated calls (the tile counter returns to
zero); a mesh with fewer tiles than the grid has CTAs; and the one-call step,
whose sensitivities run beside the pair kernel, against the separate calls."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL32, TOL64, oracle_csr

pytestmark = pytest.mark.gpu

MAT = (1.0, 1e-9, 0.3, 3.0, 0)


def to_dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def fan(n, g=None):
    """n triangles around the origin, the outer ring slightly jittered."""
    t = 2 * np.pi * np.arange(n) / n
    r = 1.0 + (0.1 * g.uniform(-1, 1, n) if g is not None else 0.0)
    coords = np.vstack([[0.0, 0.0], np.stack([r * np.cos(t), r * np.sin(t)], axis=1)])
    cells = np.array([[0, 1 + k, 1 + (k + 1) % n] for k in range(n)], np.int32)
    return coords, cells


ROUTE = {"fp32": "contract", "fp64": "pairs"}
TOL = {"fp32": (TOL32, 1e-7), "fp64": (TOL64, 1e-15)}


def check(m, cell, k, coords, cells, mat, rho, prec):
    vals = m.assemble_K(to_dev(rho))
    indptr, indices = m.pattern()
    rp, ci, v, va, ndof = oracle_csr(cell, k, coords, cells, mat, rho)
    assert np.array_equal(indptr.cpu().numpy(), rp) and np.array_equal(indices.cpu().numpy(), ci)
    err = np.abs(vals.cpu().numpy() - v)
    tol, floor = TOL[prec]
    assert np.all(err <= tol * va + floor * va.max() + 1e-300), (err / (va + 1e-300)).max()
    return vals


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_fan_past_the_staged_records(lib, k, prec):
    coords, cells = fan(150, np.random.default_rng(k))
    m = lib.Mesh("tri", k, coords, cells, *MAT, elem_prec=prec)
    assert m.routes["assembly"] == ROUTE[prec]
    rho = np.random.default_rng(7).uniform(0.001, 1.0, len(cells))
    vals = check(m, "tri", k, coords, cells, MAT, rho, prec)
    # again: the same bits (the counter of tiles was set back to zero)
    for _ in range(2):
        assert torch.equal(m.assemble_K(to_dev(rho)), vals)
    # the one-call step (sensitivities first on the second stream, the
    # contraction beside them) gives the bits of the separate calls
    u = np.random.default_rng(8).standard_normal(m.ndof)
    v2, dc2, c2 = m.step(to_dev(rho), to_dev(u))
    dc, c = m.sensitivity(to_dev(rho), to_dev(u))
    assert torch.equal(v2, vals)
    dco, so, co, sabs = oracle.sensitivity("tri", k, coords, cells, MAT, rho, u, with_abs=True)
    E0, Emin, nu, p, ps = MAT
    dE = p * rho ** (p - 1) * (E0 - Emin)
    E = Emin + rho ** p * (E0 - Emin)
    tol = TOL[prec][0]
    for d_, c_ in ((dc, c), (dc2, c2)):
        assert np.all(np.abs(d_.cpu().numpy() - dco) <= tol * dE * sabs + 1e-300)
        assert abs(c_.item() - co) <= tol * np.dot(E, sabs)
    assert torch.equal(dc2, dc)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_fan_out_of_range_moduli(lib, prec):
    """Emin = 0 with tiny and zero densities around the 150-cell centre: those
    lanes redo their pairs in FP64, reading every record from global memory."""
    mat = (1.0, 0.0, 0.3, 3.0, 0)
    coords, cells = fan(150, np.random.default_rng(3))
    m = lib.Mesh("tri", 3, coords, cells, *mat, elem_prec=prec)
    rho = np.random.default_rng(9).uniform(0.001, 1.0, len(cells))
    rho[::5] = 1e-9
    rho[1::7] = 0.0
    rho[3::11] = 1e-30
    vals = check(m, "tri", 3, coords, cells, mat, rho, prec)
    assert torch.equal(m.assemble_K(to_dev(rho)), vals)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_one_cell_and_few_tiles(lib, prec):
    """A single P3 triangle (one tile of 55 pairs' worth of lanes, most of the
    grid idle) and two triangles sharing an edge."""
    for coords, cells in ((np.array([[0.0, 0.0], [1.0, 0.1], [0.2, 0.9]]), np.array([[0, 1, 2]], np.int32)),
                          (np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]]),
                           np.array([[0, 1, 2], [0, 2, 3]], np.int32))):
        m = lib.Mesh("tri", 3, coords, cells, *MAT, elem_prec=prec)
        rho = np.linspace(0.2, 0.9, len(cells))
        vals = check(m, "tri", 3, coords, cells, MAT, rho, prec)
        assert torch.equal(m.assemble_K(to_dev(rho)), vals)
