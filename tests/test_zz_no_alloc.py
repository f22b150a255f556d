"""The allocation-free sensitivity entry point (for callers that may not
allocate device memory, e.g. inside another framework's memory pool) against
the mesh-based entry point, through the C ABI, on two calls in a row.

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


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(N, dim, shape, h, mat, rho, u, dc, c):
    n = (ctypes.c_int32 * 3)(*(list(shape) + [1] * (3 - len(shape))))
    hh = (ctypes.c_double * 3)(*(list(h) + [1.0] * (3 - len(h))))
    m = N.Material(*mat)
    return N.lib().soptx_lattice_sensitivity_noalloc(dim, n, hh, ctypes.byref(m), _ptr(rho), _ptr(u), _ptr(dc),
                                                     _ptr(c) if c is not None else None,
                                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("dim,shape,h", [(3, (13, 5, 4), (1.0, 1.0, 1.0)), (3, (7, 6, 3), (0.5, 1.25, 2.0)),
                                         (2, (21, 9), (1.0, 1.0)), (2, (9, 4), (2.0, 0.5))])
def test_noalloc_matches_mesh_entry_point(lib, dim, shape, h):
    from paper_2505_02438_gb300 import _native as N
    coords, cells = W.structured_hex(*shape) if dim == 3 else W.structured_quad(*shape)
    coords = coords * np.array(h)
    cell = "hex" if dim == 3 else "quad"
    mat = (1.0, 1e-9, 0.3, 3.0, 0)
    mesh = lib.Mesh(cell, 1, coords, cells, *mat)
    assert mesh.path == "lattice"
    g = np.random.default_rng(31)
    for call in range(2):
        rho = g.uniform(0.001, 1.0, len(cells))
        u = g.standard_normal(mesh.ndof)
        rho_d = torch.as_tensor(rho, device="cuda")
        u_d = torch.as_tensor(u, device="cuda")
        dc_ref, c_ref = mesh.sensitivity(rho_d, u_d)
        dc = torch.full((len(cells),), np.nan, dtype=torch.float64, device="cuda")
        c = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        assert _noalloc(N, dim, shape, h, mat, rho_d, u_d, dc, c) == 0, N.lib().soptx_last_error()
        torch.cuda.synchronize()
        # tolerance of the parity tests: 1e-12 of |E'| sum_ab |u_a K_ab u_b|
        _, _, _, sabs = oracle.sensitivity(cell, 1, coords, cells, mat, rho, u, with_abs=True)
        dE = mat[3] * rho ** (mat[3] - 1) * (mat[0] - mat[1])
        E = mat[1] + rho ** mat[3] * (mat[0] - mat[1])
        err = np.abs(dc.cpu().numpy() - dc_ref.cpu().numpy())
        assert np.all(err <= TOL64 * dE * sabs), (call, err.max())
        assert abs(c.item() - c_ref.item()) <= TOL64 * np.dot(E, sabs), call


def test_noalloc_rejects_lattices_beyond_the_limit(lib):
    from paper_2505_02438_gb300 import _native as N
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = _noalloc(N, 3, (2049, 2048, 2), (1.0, 1.0, 1.0), (1.0, 1e-9, 0.3, 3.0, 0), t, t, t, None)
    assert rc == 1
    assert b"allocation-free limit" in N.lib().soptx_last_error()
