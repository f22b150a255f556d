"""The allocation-free sensitivity entry point (for callers that may not
allocate device memory, e.g. inside another framework's memory pool) through
the C ABI, on two calls in a row: against the oracle's dc and c directly, and
against the mesh-based entry point.

Kept in a file of its own that sorts last, so that a run stopping at the first
failure has run every other test before it."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from helpers import TOL64
from paper_2505_02438_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MAT = (1.0, 1e-9, 0.3, 3.0, 0)
# the entry point's fixed scratch holds one partial of c per 1024 cells, 8192 of them
MAX_CELLS = 8192 * 1024


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(N, dim, shape, h, mat, rho, u, dc, c):
    n = (ctypes.c_int32 * 3)(*(list(shape) + [1] * (3 - len(shape))))
    hh = (ctypes.c_double * 3)(*(list(h) + [1.0] * (3 - len(h))))
    m = N.Material(*mat)
    return N.lib().soptx_lattice_sensitivity_noalloc(dim, n, hh, ctypes.byref(m), _ptr(rho), _ptr(u), _ptr(dc),
                                                     _ptr(c) if c is not None else None,
                                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _lattice(dim, shape, h):
    coords, cells = W.structured_hex(*shape) if dim == 3 else W.structured_quad(*shape)
    return coords * np.array(h), cells, ("hex" if dim == 3 else "quad")


def _scales(rho, sabs):
    dE = MAT[3] * rho ** (MAT[3] - 1) * (MAT[0] - MAT[1])
    E = MAT[1] + rho ** MAT[3] * (MAT[0] - MAT[1])
    return dE * sabs, np.dot(E, sabs)


# one block (<= 1024 cells), several blocks with a ragged last one, anisotropic boxes
@pytest.mark.parametrize("dim,shape,h", [(3, (13, 5, 4), (1.0, 1.0, 1.0)), (3, (7, 6, 3), (0.5, 1.25, 2.0)),
                                         (3, (60, 20, 20), (1.0, 1.0, 1.0)), (3, (23, 11, 7), (0.5, 1.25, 2.0)),
                                         (2, (21, 9), (1.0, 1.0)), (2, (9, 4), (2.0, 0.5)),
                                         (2, (800, 400), (1.0, 1.0)), (2, (203, 97), (2.0, 0.5))])
def test_noalloc_matches_oracle_and_mesh_entry_point(lib, dim, shape, h):
    from paper_2505_02438_gb300 import _native as N
    coords, cells, cell = _lattice(dim, shape, h)
    mesh = lib.Mesh(cell, 1, coords, cells, *MAT)
    assert mesh.path == "lattice"
    g = np.random.default_rng(31 + len(cells))
    for call in range(2):
        rho = g.uniform(0.001, 1.0, len(cells))
        u = g.standard_normal(mesh.ndof)
        if call == 1:
            u += 50.0   # a large rigid translation on top: its Walsh mode must not leak into dc
        rho_d = torch.as_tensor(rho, device="cuda")
        u_d = torch.as_tensor(u, device="cuda")
        dc = torch.full((len(cells),), np.nan, dtype=torch.float64, device="cuda")
        c = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        assert _noalloc(N, dim, shape, h, MAT, rho_d, u_d, dc, c) == 0, N.lib().soptx_last_error()
        dc_mesh, c_mesh = mesh.sensitivity(rho_d, u_d)
        torch.cuda.synchronize()
        dco, _, co, sabs = oracle.sensitivity(cell, 1, coords, cells, MAT, rho, u, with_abs=True)
        tol_dc, tol_c = _scales(rho, sabs)
        got = dc.cpu().numpy()
        err = np.abs(got - dco)
        assert np.all(err <= TOL64 * tol_dc), (call, err.max())
        assert abs(c.item() - co) <= TOL64 * tol_c, (call, c.item(), co)
        # and the mesh entry point, within the same tolerance
        assert np.all(np.abs(got - dc_mesh.cpu().numpy()) <= TOL64 * tol_dc), call
        assert abs(c.item() - c_mesh.item()) <= TOL64 * tol_c, call


def test_noalloc_at_the_cell_limit(lib):
    """8,388,608 cells (every slot of the scratch array in use), two calls:
    sampled cells against the oracle, c against the fixed-order sum of the
    call's own strain energies."""
    from paper_2505_02438_gb300 import _native as N
    shape, h = (2048, 2048, 2), (1.0, 0.5, 2.0)
    coords, cells, cell = _lattice(3, shape, h)
    assert len(cells) == MAX_CELLS
    ndof = 3 * len(coords)
    g = np.random.default_rng(77)
    sel = np.sort(g.choice(len(cells), 3000, replace=False))
    sel = np.unique(np.concatenate([sel, [0, 1023, 1024, len(cells) - 1025, len(cells) - 1]])).astype(np.int64)
    dc = torch.empty(len(cells), dtype=torch.float64, device="cuda")
    c = torch.empty(1, dtype=torch.float64, device="cuda")
    for call in range(2):
        rho = g.uniform(0.001, 1.0, len(cells))
        u = g.standard_normal(ndof)
        rho_d = torch.as_tensor(rho, device="cuda")
        u_d = torch.as_tensor(u, device="cuda")
        dc.fill_(np.nan)
        c.fill_(np.nan)
        assert _noalloc(N, 3, shape, h, MAT, rho_d, u_d, dc, c) == 0, N.lib().soptx_last_error()
        torch.cuda.synchronize()
        got = dc.cpu().numpy()
        assert np.all(np.isfinite(got))
        dco, _, _, sabs = oracle.sensitivity(cell, 1, coords, cells, MAT, rho, u, sel=sel, with_abs=True)
        tol_dc, _ = _scales(rho[sel], sabs)
        assert np.all(np.abs(got[sel] - dco) <= TOL64 * tol_dc), call
        # s_e = u_e^T K u_e >= 0 from dc; c = sum_e E_e s_e (the partials of all 8192 blocks)
        dE = MAT[3] * rho ** (MAT[3] - 1) * (MAT[0] - MAT[1])
        E = MAT[1] + rho ** MAT[3] * (MAT[0] - MAT[1])
        s = -got / dE
        ref = float(np.sum(E * s))
        assert abs(c.item() - ref) <= 1e-12 * abs(ref), (call, c.item(), ref)
    del rho_d, u_d, dc, c
    torch.cuda.empty_cache()


def test_noalloc_rejects_lattices_beyond_the_limit(lib):
    from paper_2505_02438_gb300 import _native as N
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = _noalloc(N, 3, (2049, 2048, 2), (1.0, 1.0, 1.0), MAT, t, t, t, None)
    assert rc == 1
    assert b"allocation-free limit" in N.lib().soptx_last_error()
