"""The steps after the sensitivities on the GPU against the oracle: the
filters and the density filter's chain rule, the Heaviside projection, the OC
update, and the whole optimisation loop of the paper's 3D cantilever
(Sec. 5.4) against the oracle's stored trajectory and the paper's printed
result."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2505_02438_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float64), device="cuda")


MESHES = {
    "tet": lambda: ("tet", *W.kuhn_tets(5, 4, 3, 0.15, np.random.default_rng(1)), 1.4),
    "tri": lambda: ("tri", *W.triangle_grid(14, 9, 0.2, np.random.default_rng(2)), 2.5),
    "quadj": lambda: ("quad", *W.quad_grid(12, 7, 0.2, np.random.default_rng(3)), 1.7),
    "hex": lambda: ("hex", *W.structured_hex(9, 5, 4), 1.5),
}


@pytest.mark.parametrize("name", sorted(MESHES))
def test_filters_match_oracle(lib, name):
    from paper_2505_02438_gb300.optim import Filter, cell_centroids_volumes
    cell, coords, cells, rmin = MESHES[name]()
    cen, vol = cell_centroids_volumes(cell, coords, cells)
    H = oracle.filter_weights(cen, rmin)
    flt = Filter(cen, vol, rmin)
    assert flt.nnz == H.nnz
    g = np.random.default_rng(7)
    rho = g.uniform(0.0, 1.0, len(cells))
    dc = -g.uniform(0.0, 3.0, len(cells))
    x = g.uniform(0.0, 1.0, len(cells))
    gr = g.standard_normal(len(cells))
    np.testing.assert_allclose(flt.sensitivity(dev(rho), dev(dc)).cpu().numpy(),
                               oracle.sensitivity_filter(H, rho, dc), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(flt.density(dev(x)).cpu().numpy(), oracle.density_filter(H, vol, x),
                               rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(flt.density_grad(dev(gr)).cpu().numpy(), oracle.density_filter_grad(H, vol, gr),
                               rtol=1e-12, atol=1e-13 * np.abs(gr).max())
    flt.close()


def test_heaviside_matches_oracle(lib):
    from paper_2505_02438_gb300.optim import heaviside
    x = np.random.default_rng(8).uniform(0, 1, 1000)
    for beta in (1.0, 16.0):
        y, dy = heaviside(dev(x), beta, want_derivative=True)
        yo, dyo = oracle.heaviside(x, beta)
        np.testing.assert_allclose(y.cpu().numpy(), yo, rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(dy.cpu().numpy(), dyo, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("n,eta", [(1000, 0.5), (33000, 0.5), (5000, 1.0), (777, 0.3)])
def test_oc_update_matches_oracle(lib, n, eta):
    from paper_2505_02438_gb300.optim import oc_update
    g = np.random.default_rng(n)
    rho = g.uniform(0.0, 1.0, n)
    dc = -g.uniform(0.0, 4.0, n)
    vol = g.uniform(0.5, 1.5, n)
    new, st = oc_update(dev(rho), dev(dc), dev(vol), dev(vol), 0.35, eta=eta)
    want, lam = oracle.oc_update(rho, dc, vol, vol, 0.35, eta=eta)
    assert st["lam"] == pytest.approx(lam, rel=1e-15)
    np.testing.assert_allclose(new.cpu().numpy(), want, rtol=1e-13, atol=1e-15)
    assert st["change"] == pytest.approx(np.abs(want - rho).max(), rel=1e-13)
    assert st["vol_frac"] == pytest.approx(np.dot(vol, want) / vol.sum(), rel=1e-13)


def test_oc_loop_reproduces_the_papers_3d_cantilever(lib):
    """The whole loop on the device (assembly, constrained CG, sensitivities,
    filter, OC) on the paper's 3D cantilever: the oracle's per-iteration
    compliance, its 54 iterations and the paper's c = 2063.5625."""
    from paper_2505_02438_gb300.optim import cell_centroids_volumes, oc_loop
    with open(os.path.join(GOLDEN, "paper_cantilever3d.json")) as fh:
        paper = json.load(fh)["60x20x4"]
    with open(os.path.join(GOLDEN, "cantilever3d_60x20x4_oc.json")) as fh:
        stored = json.load(fh)
    wl, fixed, f = W.cantilever_3d_oc(60, 20, 4)
    m = lib.Mesh.from_workload(wl)
    cen, vol = cell_centroids_volumes("hex", wl.coords, wl.cells)
    r = oc_loop(m, fixed, f, paper["rmin"], paper["volfrac"], vol, cen, cg_rtol=1e-10)
    c = [h[0] for h in r["history"]]
    assert len(c) == paper["iterations"] == len(stored["c"])
    np.testing.assert_allclose(c, stored["c"], rtol=1e-7)
    assert abs(c[-1] - paper["c"]) <= 5e-5
