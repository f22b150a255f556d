"""The C ABI without a GPU: the in-tree library loads, exports every symbol the
public headers declare, and its host-side numbering / CSR pattern equals the
oracle's, bit for bit."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle
from helpers import relabel, small_cases
from paper_2505_02438_gb300 import build, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    build.build_library()
    from paper_2505_02438_gb300 import _native
    return _native


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(soptx_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol(native):
    L = ctypes.CDLL(native.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the binding declares a signature for each of them
    assert set(names) <= set(native.SIGNATURES), set(names) - set(native.SIGNATURES)


def test_version_and_error_string(native):
    assert b"sm_103a" in native.lib().soptx_version()
    assert isinstance(native.lib().soptx_last_error(), bytes)


@pytest.mark.parametrize("name,cell,k,coords,cells", small_cases(), ids=[c[0] for c in small_cases()])
def test_host_pattern_equals_oracle(native, name, cell, k, coords, cells):
    from paper_2505_02438_gb300.api import host_plan
    pl = host_plan(cell, k, coords, cells)
    rp, ci, v, ndof = oracle.assemble(cell, k, coords, cells, (1, 1e-9, .3, 3, 0), np.ones(len(cells)))
    assert pl["ndof"] == ndof
    assert np.array_equal(pl["indptr"], rp)
    assert np.array_equal(pl["indices"], ci)
    cn, nn = oracle.number(cell, k, len(coords), cells)
    for a, b in zip(pl["cell_nodes"], cn):
        assert sorted(a) == sorted(b)


@pytest.mark.parametrize("cell,k", [("tri", 3), ("tet", 2), ("tet", 3), ("quad", 2), ("hex", 2), ("hex", 3)])
def test_host_pattern_relabelled_vertices(native, cell, k):
    from paper_2505_02438_gb300.api import host_plan
    g = np.random.default_rng(5)
    mk = {"tri": lambda: W.triangle_grid(5, 4, 0.2, g), "tet": lambda: W.kuhn_tets(3, 2, 2, 0.1, g),
          "quad": lambda: W.structured_quad(4, 3), "hex": lambda: W.structured_hex(2, 2, 2)}[cell]
    coords, cells = relabel(*mk(), 11)
    pl = host_plan(cell, k, coords, cells)
    rp, ci, v, ndof = oracle.assemble(cell, k, coords, cells, (1, 1e-9, .3, 3, 0), np.ones(len(cells)))
    assert np.array_equal(pl["indptr"], rp) and np.array_equal(pl["indices"], ci)


def test_paths_selected():
    from paper_2505_02438_gb300.api import host_plan
    assert host_plan("hex", 1, *W.structured_hex(4, 3, 2))["path"] == "lattice"
    assert host_plan("quad", 1, *W.structured_quad(4, 3))["path"] == "lattice"
    assert host_plan("hex", 1, *relabel(*W.structured_hex(4, 3, 2), 1))["path"] == "uniform"
    assert host_plan("hex", 2, *W.structured_hex(4, 3, 2))["path"] == "uniform"
    assert host_plan("tri", 1, *W.triangle_grid(4, 3, 0.2, np.random.default_rng(0)))["path"] == "cached"


def test_distorted_tensor_cells_take_the_cached_path():
    """General (non-affine) quads / hexes are integrated by Gauss quadrature
    per cell: accepted, numbered like any mesh, never lattice or uniform."""
    from paper_2505_02438_gb300.api import host_plan
    g = np.random.default_rng(0)
    pl = host_plan("quad", 2, *W.quad_grid(5, 4, 0.2, g))
    assert pl["path"] == "cached" and pl["ndof"] == 2 * 11 * 9
    assert host_plan("hex", 1, *W.hex_grid(3, 3, 2, 0.15, g))["path"] == "cached"


def test_empty_mesh_plan():
    from paper_2505_02438_gb300.api import host_plan
    pl = host_plan("tri", 2, np.zeros((3, 2)), np.zeros((0, 3), np.int32))
    assert pl["ndof"] == 6 and pl["nnz"] == 0 and np.all(pl["indptr"] == 0)


@pytest.mark.parametrize("bad,msg", [
    (lambda c, cl: (c, np.where(cl == 0, 10 ** 6, cl)), "out of range"),
    (lambda c, cl: (c, np.concatenate([cl[:, :1], cl[:, :1], cl[:, 2:]], 1)), "repeats a vertex"),
    (lambda c, cl: (np.where(np.arange(len(c))[:, None] == 6, c + 1.8, c), cl), "inverted or degenerate"),
])
def test_invalid_meshes_rejected(bad, msg):
    from paper_2505_02438_gb300 import _native as N
    from paper_2505_02438_gb300.api import host_plan
    coords, cells = bad(*W.structured_quad(4, 3))
    with pytest.raises(N.SoptxError) as ei:
        host_plan("quad", 1, coords, cells)
    assert ei.value.code == 1 and msg in str(ei.value)


def test_degenerate_simplex_rejected():
    from paper_2505_02438_gb300 import _native as N
    from paper_2505_02438_gb300.api import host_plan
    coords = np.array([[0, 0], [1, 0], [2, 0.0]])
    with pytest.raises(N.SoptxError, match="degenerate"):
        host_plan("tri", 1, coords, np.array([[0, 1, 2]], np.int32))


def test_wrong_dimension_and_order_rejected():
    from paper_2505_02438_gb300 import _native as N
    from paper_2505_02438_gb300.api import host_plan
    c, cl = W.structured_quad(2, 2)
    with pytest.raises(N.SoptxError, match="order"):
        host_plan("quad", 4, c, cl)
    with pytest.raises(N.SoptxError, match="dim"):
        host_plan("hex", 1, c, cl)


def test_null_mesh_calls_return_einval(native):
    """Every entry point that takes a mesh refuses NULL with SOPTX_EINVAL
    before touching the device."""
    L = native.lib()
    EINVAL = 1
    p = ctypes.c_void_p(0)
    assert L.soptx_assemble_K(None, p, p, p) == EINVAL
    assert L.soptx_sensitivity(None, p, p, p, p, p) == EINVAL
    assert L.soptx_assemble_and_sensitivity(None, p, p, p, p, p, p) == EINVAL
    assert L.soptx_step_host(None, p, p, p, p, p, p) == EINVAL
    assert L.soptx_compliance_vjp(None, p, p, p, p, p, p) == EINVAL
    assert b"NULL" in L.soptx_last_error()


def test_traffic_records_are_keyed_on_kernel_workload_and_precision():
    """bench.py reports ncu traffic only for the kernel, workload and element
    precision it was captured on, and only while the kernel source is
    unchanged."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    rec = os.path.join(ROOT, "profiles", "traffic.txt")
    lines = [dict(x.split("=", 1) for x in ln.split() if "=" in x) for ln in open(rec) if ln.startswith("kernel=")]
    assert lines
    src = {"k_lattice_assemble3": "lattice.cu", "k_lattice_assemble2": "lattice.cu", "k_lattice_sens": "lattice.cu",
           "k_gather_rows": "gather.cu", "k_gather_nodes": "gather.cu", "k_contract_rows": "contract.cu",
           "k_contract_pairs": "contract.cu", "k_strain_hex_sf": "contract.cu",
           "k_strain_energy": "contract.cu", "k_spmv": "solve.cu", "k_simp_df": "lattice.cu", "k_prep": "gather.cu",
           "k_sens_finalize": "gather.cu"}
    for kv in lines:
        f = src[kv["kernel"]]
        got = bench.traffic_record(f, kv["kernel"], kv["workload"], kv.get("prec", "fp64"))
        if kv["source_sha"] == bench.kernel_source_sha(f):
            assert got == float(kv["dram_bytes_per_launch"])
        # never another workload's or precision's figure
        assert bench.traffic_record(f, kv["kernel"], kv["workload"] + "_other", kv.get("prec", "fp64")) is None
    assert bench.traffic_record("gather.cu", "k_gather_rows", "tet_p2_60x20x20", "fp16") is None


@pytest.mark.parametrize("mk,cell,k,nc,ndof,nnz", [
    (lambda: W.mbb_q4(60, 20), "quad", 1, 1200, 2562, 44164),
    (lambda: W.cantilever_hex(120, 40, 40), "hex", 1, 192000, 610203, 47568609),
    (lambda: W.jittered_tri(400, 200), "tri", 3, 160000, 1443602, 48996004),
    (lambda: W.jittered_tet(60, 20, 20), "tet", 2, 144000, 610203, 50846409),
    (lambda: W.mbb_q4(800, 400), "quad", 1, 320000, 642402, 11534404),
    (lambda: W.cantilever_hex(30, 10, 10), "hex", 1, 3000, 11253, 787059),
], ids=["q4_60x20", "hex_120x40x40", "tri_p3_400x200", "tet_p2_60x20x20", "q4_800x400", "hex_30x10x10"])
def test_standard_workload_sizes(native, mk, cell, k, nc, ndof, nnz):
    """The synthetic workloads have the cell, dof and nonzero counts of the
    specified configurations (host-side plan, sizes only)."""
    wl = mk()
    assert wl.cell == cell and wl.order == k and len(wl.cells) == nc
    coords = np.ascontiguousarray(wl.coords, np.float64)
    cells = np.ascontiguousarray(wl.cells, np.int32)
    nd, nz, nb, path = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    native.check(native.lib().soptx_host_plan(coords.shape[1], native.CELL[cell], k, coords.shape[0],
                                              coords.ctypes.data_as(ctypes.c_void_p), cells.shape[0],
                                              cells.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nd),
                                              ctypes.byref(nz), ctypes.byref(nb), ctypes.byref(path), None, None,
                                              None))
    assert (nd.value, nz.value) == (ndof, nnz)
