"""Complete parity at the full workload sizes: every CSR index, every CSR value,
every dc and c of the GPU step against the oracle's (computed by the oracle
unchanged over row and cell ranges in a spawned process pool), in the launch
configurations the benchmark times.

* the 3D cantilever box 120 x 40 x 40 (box lattice), P3 triangles 400 x 200 and
  Kuhn P2 tetrahedra 60 x 20 x 20 (general meshes), FP64 and FP32 element
  matrices;
* Q2 hexahedra 40 x 14 x 14 (36.9 M nonzeros) and Q3 hexahedra 26 x 9 x 9
  (65.1 M nonzeros), as boxes and with jittered interior vertices;
* Q4 800 x 400 and 803 x 397, sizes at which the 2D lattice kernel takes
  48-node chunks of 16 passes (803 x 397: chunks straddle lattice rows), by the
  one-call step and by the separate calls."""
import numpy as np
import pytest
import torch

from helpers import TOL32, TOL64, oracle_full_parallel
from paper_2505_02438_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WORKLOADS = {
    "hex_120x40x40": lambda: W.cantilever_hex(120, 40, 40),
    "tri_p3_400x200": lambda: W.jittered_tri(400, 200),
    "tet_p2_60x20x20": lambda: W.jittered_tet(60, 20, 20),
    "q4_800x400": lambda: W.mbb_q4(800, 400),
    "q4_803x397": lambda: W.mbb_q4(803, 397),
    # Q2 / Q3 hexahedra at scale: 27- and 64-node cells, affine boxes (one shared
    # element matrix) and jittered general trilinear cells (Gauss rule per cell)
    "hexq2_40x14x14": lambda: W.cantilever_hex(40, 14, 14, order=2),
    "hexq2j_40x14x14": lambda: W.jittered_hex(40, 14, 14, order=2),
    "hexq3_26x9x9": lambda: W.cantilever_hex(26, 9, 9, order=3),
    "hexq3j_26x9x9": lambda: W.jittered_hex(26, 9, 9, order=3),
}
_ORACLE = {}


def reference(name, lib):
    """(workload, u, oracle results), the oracle run once per workload."""
    if name not in _ORACLE:
        _ORACLE.clear()   # one full-size reference held at a time
        wl = WORKLOADS[name]()
        plan = lib.host_plan(wl.cell, wl.order, wl.coords, wl.cells)
        u = wl.displacement(plan["ndof"])
        _ORACLE[name] = (wl, u, oracle_full_parallel(wl.cell, wl.order, wl.coords, wl.cells, wl.mat, wl.rho, u,
                                                     plan["ndof"]))
    return _ORACLE[name]


def compare(name, prec, wl, u, ref, indptr, indices, vals, dc, c):
    rp, ci, v, va, dco, so, sa = ref
    tol = TOL64 if prec == "fp64" else TOL32
    assert np.array_equal(indptr, rp), name
    assert np.array_equal(indices, ci), name
    floor = (1e-15 if prec == "fp64" else 1e-7) * va.max()
    err = np.abs(vals - v)
    bad = np.nonzero(err > tol * va + floor)[0]
    assert len(bad) == 0, (name, prec, len(bad), int(bad[0]) if len(bad) else None)
    E0, Emin, nu, p, ps = wl.mat
    dE = p * wl.rho ** (p - 1) * (E0 - Emin)
    E = Emin + wl.rho ** p * (E0 - Emin)
    derr = np.abs(dc - dco)
    assert np.all(derr <= tol * dE * sa), (name, prec, float((derr / (dE * sa)).max()))
    co = float(np.dot(E, so))
    assert abs(c - co) <= tol * np.dot(E, sa), (name, prec, c, co)
    rel = err / (va + floor / tol)
    print("%s %s: %d values, max err/scale %.3e; %d cells, max dc err/scale %.3e" % (
        name, prec, len(v), rel.max(), len(dc), (derr / (dE * sa)).max()))


@pytest.mark.parametrize("name,prec", [("hex_120x40x40", "fp64"), ("tri_p3_400x200", "fp64"),
                                       ("tri_p3_400x200", "fp32"), ("tet_p2_60x20x20", "fp64"),
                                       ("tet_p2_60x20x20", "fp32"), ("hexq2_40x14x14", "fp64"),
                                       ("hexq2_40x14x14", "fp32"), ("hexq2j_40x14x14", "fp64"),
                                       ("hexq3_26x9x9", "fp64"), ("hexq3j_26x9x9", "fp64")])
def test_full_size_complete_parity(lib, name, prec):
    wl, u, ref = reference(name, lib)
    m = lib.Mesh.from_workload(wl, elem_prec=prec)
    rho = torch.as_tensor(wl.rho, device="cuda")
    ud = torch.as_tensor(u, device="cuda")
    vals, dc, c = m.step(rho, ud)
    indptr, indices = m.pattern()
    torch.cuda.synchronize()
    compare(name, prec, wl, u, ref, indptr.cpu().numpy(), indices.cpu().numpy(), vals.cpu().numpy(),
            dc.cpu().numpy(), c.item())
    m.close()


@pytest.mark.parametrize("name", ["q4_800x400", "q4_803x397"])
def test_2d_lattice_long_chunks_complete_parity(lib, name):
    wl, u, ref = reference(name, lib)
    m = lib.Mesh.from_workload(wl)
    assert m.path == "lattice"
    rho = torch.as_tensor(wl.rho, device="cuda")
    ud = torch.as_tensor(u, device="cuda")
    indptr, indices = m.pattern()
    ip, ix = indptr.cpu().numpy(), indices.cpu().numpy()
    # the one-call step (sensitivities on the mesh's second stream) ...
    vals, dc, c = m.step(rho, ud)
    torch.cuda.synchronize()
    compare(name + " step", "fp64", wl, u, ref, ip, ix, vals.cpu().numpy(), dc.cpu().numpy(), c.item())
    # ... and the separate calls, into fresh buffers
    vals2 = m.assemble_K(rho)
    dc2, c2 = m.sensitivity(rho, ud)
    torch.cuda.synchronize()
    compare(name + " separate", "fp64", wl, u, ref, ip, ix, vals2.cpu().numpy(), dc2.cpu().numpy(), c2.item())
    m.close()
