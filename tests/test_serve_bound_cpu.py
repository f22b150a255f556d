"""The serving admission bound (soptx_serve_mesh_bytes_bound), checked without a
GPU: it covers the largest device arrays of a mesh as mesh creation sizes them
on the host -- the element-matrix cache, the CSR indices and the pair kernel's
tables (records padded per tile, pairs padded to whole chunks, and in 2D with
FP64 element matrices each record's cached 2 x 2 block) -- on triangles and
affine quadrilaterals of every order, both element precisions, and a 150-cell
fan (the widest padding per pair)."""
import numpy as np
import pytest

from paper_2505_02438_gb300 import _native as N, build, workloads as W


@pytest.fixture(scope="module", autouse=True)
def native():
    build.build_library()


def rectangles(nx, ny):
    """Axis-aligned rectangles of varying width: affine cells, not a uniform mesh."""
    coords, cells = W.structured_quad(nx, ny)
    coords = coords.copy()
    coords[:, 0] += 0.01 * coords[:, 0] ** 2
    return coords, cells


def fan(n):
    t = 2 * np.pi * np.arange(n) / n
    coords = np.vstack([[0.0, 0.0], np.stack([np.cos(t), np.sin(t)], axis=1)])
    return coords, np.array([[0, 1 + k, 1 + (k + 1) % n] for k in range(n)], np.int32)


def largest_arrays(cell, k, coords, cells, prec):
    """Bytes of the element-matrix cache, the CSR indices and the pair tables."""
    from paper_2505_02438_gb300.api import host_pair_tables, host_plan
    pl = host_plan(cell, k, coords, cells)
    d, nc = coords.shape[1], len(cells)
    ldof = d * pl["nb"]
    b = nc * ldof * ldof * (8 if prec == "fp64" else 4) + 4 * pl["nnz"]
    T = host_pair_tables(cell, k, coords, cells, prec == "fp64")
    if T is not None:
        nchunks = (T["n_tiles"] + 7) // 8
        nrec = len(T["record_cell"])
        b += 4 * (nchunks * 8 + 16) + 3 * 4 * nchunks * 8 * 32 + 6 * nrec + (32 * nrec if prec == "fp64" else 0)
    return b


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("cell,k,mk", [
    ("tri", 1, lambda: W.triangle_grid(60, 40, 0.2, np.random.default_rng(1))),
    ("tri", 2, lambda: W.triangle_grid(40, 30, 0.2, np.random.default_rng(2))),
    ("tri", 3, lambda: W.triangle_grid(40, 20, 0.2, np.random.default_rng(3))),
    ("quad", 1, lambda: rectangles(60, 30)),
    ("quad", 2, lambda: rectangles(40, 20)),
    ("quad", 3, lambda: rectangles(30, 20)),
    ("tri", 3, lambda: fan(150)),
], ids=["tri1", "tri2", "tri3", "quad1", "quad2", "quad3", "fan150"])
def test_bound_covers_cache_indices_and_pair_tables(cell, k, mk, prec):
    from paper_2505_02438_gb300.serve import mesh_bytes_bound
    coords, cells = mk()
    wl = W.Workload("t", cell, k, coords, cells, elem_prec=prec)
    assert mesh_bytes_bound(wl) >= largest_arrays(cell, k, coords, cells, prec)


def test_malformed_request_rejected():
    import ctypes
    from paper_2505_02438_gb300.serve import _mesh_request
    coords, cells = W.triangle_grid(4, 3, 0.0)
    r = _mesh_request(W.Workload("t", "tri", 1, coords, cells), coords, cells)
    r.order = 4
    b = ctypes.c_int64()
    assert N.lib().soptx_serve_mesh_bytes_bound(ctypes.byref(r), ctypes.byref(b)) == 1
    assert N.lib().soptx_serve_mesh_bytes_bound(None, ctypes.byref(b)) == 1


def test_ids_out_of_range_are_skipped():
    """The bound reads the cell array before mesh creation validates it: ids
    outside [0, n_vertices) are skipped there (creation then rejects the mesh)."""
    from paper_2505_02438_gb300.serve import mesh_bytes_bound
    coords, cells = W.triangle_grid(6, 4, 0.0)
    bad = cells.copy()
    bad[0, 0], bad[1, 2] = 10 ** 6, -5
    good = mesh_bytes_bound(W.Workload("t", "tri", 2, coords, cells))
    assert 0 < mesh_bytes_bound(W.Workload("t", "tri", 2, coords, bad)) <= good
