"""The grouped one-call step (soptx_assemble_and_sensitivity_group): small 2D and
3D box lattices share one launch, a cluster of CTAs each.  Each mesh's K, dc and
c must be bitwise those of its own step (the same arithmetic in the same order),
and therefore match the oracle; other meshes in the group take the ordinary
call."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL64, oracle_csr
from paper_2505_02438_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MAT = (1.0, 1e-9, 0.3, 3.0, 0)


def to_dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def inputs(m, seed):
    g = np.random.default_rng(seed)
    return g.uniform(0.001, 1.0, m.n_cells), g.standard_normal(m.ndof)


# Q4 and hex Q1 boxes: one cell, one row and one column of cells, ragged node
# chunks, exactly the largest grouped size (4096 cells in 2D, 1024 in 3D); then
# meshes that are not grouped (4097 and 1088 cells, distorted quads and hexes)
GROUPED = [(1, 1), (7, 1), (1, 9), (60, 20), (17, 9), (64, 64), (128, 32), (3, 50)]
GROUPED3 = [(1, 1, 1), (5, 4, 3), (16, 8, 8), (10, 10, 10), (17, 9, 5), (1, 1, 40)]
ORDINARY = [("quad", lambda: W.structured_quad(4097, 1)), ("hex", lambda: W.structured_hex(17, 8, 8)),
            ("quad", lambda: W.quad_grid(9, 6, jitter=0.2, g=np.random.default_rng(3))),
            ("hex", lambda: W.hex_grid(4, 3, 2, jitter=0.15, g=np.random.default_rng(4)))]


def make_meshes(lib, mat=MAT):
    ms = []
    for nx, ny in GROUPED:
        c, cl = W.structured_quad(nx, ny)
        ms.append(("quad", c, cl, lib.Mesh("quad", 1, c, cl, *mat)))
    for nx, ny, nz in GROUPED3:
        c, cl = W.structured_hex(nx, ny, nz)
        ms.append(("hex", c, cl, lib.Mesh("hex", 1, c, cl, *mat)))
    for cell, mk in ORDINARY:
        c, cl = mk()
        ms.append((cell, c, cl, lib.Mesh(cell, 1, c, cl, *mat)))
    return ms


def test_group_is_bitwise_each_meshs_own_step(lib):
    from paper_2505_02438_gb300 import step_group
    ms = make_meshes(lib)
    assert all(m.path == "lattice" for _, _, _, m in ms[:len(GROUPED) + len(GROUPED3)])
    ins = [inputs(m, 10 + k) for k, (_, _, _, m) in enumerate(ms)]
    rhos = [to_dev(r) for r, _ in ins]
    us = [to_dev(u) for _, u in ins]
    got = step_group([m for *_, m in ms], rhos, us)
    torch.cuda.synchronize()
    for (cell, c, cl, m), rho, u, (vals, dc, cc) in zip(ms, rhos, us, got):
        v1, d1, c1 = m.step(rho, u)
        assert torch.equal(vals, v1) and torch.equal(dc, d1) and torch.equal(cc, c1), (cell, m.n_cells)
    # twice in a row (the out-of-range generation and the sum's ticket reset)
    again = step_group([m for *_, m in ms], rhos, us)
    for (vals, dc, cc), (v2, d2, c2) in zip(got, again):
        assert torch.equal(vals, v2) and torch.equal(dc, d2) and torch.equal(cc, c2)


def test_group_matches_oracle(lib):
    from paper_2505_02438_gb300 import step_group
    shapes = [("quad", W.structured_quad(60, 20)), ("quad", W.structured_quad(64, 64)),
              ("quad", W.structured_quad(5, 3)), ("hex", W.structured_hex(12, 8, 6)),
              ("hex", W.structured_hex(3, 2, 2))]
    meshes, rhos, us, data = [], [], [], []
    for k, (cell, (c, cl)) in enumerate(shapes):
        m = lib.Mesh(cell, 1, c, cl, *MAT)
        rho, u = inputs(m, 40 + k)
        meshes.append(m)
        rhos.append(to_dev(rho))
        us.append(to_dev(u))
        data.append((cell, c, cl, rho, u))
    got = step_group(meshes, rhos, us)
    for (cell, c, cl, rho, u), m, (vals, dc, cc) in zip(data, meshes, got):
        rp, ci, v, va, _ = oracle_csr(cell, 1, c, cl, MAT, rho)
        assert np.all(np.abs(vals.cpu().numpy() - v) <= TOL64 * va + 1e-15 * va.max())
        dco, so, co, sabs = oracle.sensitivity(cell, 1, c, cl, MAT, rho, u, with_abs=True)
        E0, Emin, nu, p, ps = MAT
        dE = p * rho ** (p - 1) * (E0 - Emin)
        E = Emin + rho ** p * (E0 - Emin)
        assert np.all(np.abs(dc.cpu().numpy() - dco) <= TOL64 * dE * sabs + 1e-300)
        assert abs(cc.item() - co) <= TOL64 * np.dot(E, sabs)


def test_group_out_of_range_moduli(lib):
    """Emin = 0 with tiny and zero densities: the moduli kernel's FP64 rows for
    the nodes around those cells, in the grouped kernel as in the single step."""
    from paper_2505_02438_gb300 import step_group
    mat = (1.0, 0.0, 0.3, 3.0, 0)
    meshes, rhos, us = [], [], []
    shapes = [("quad", W.structured_quad(9, 7)), ("quad", W.structured_quad(33, 20)),
              ("hex", W.structured_hex(5, 4, 3)), ("hex", W.structured_hex(14, 10, 9))]
    for k, (cell, (c, cl)) in enumerate(shapes):
        m = lib.Mesh(cell, 1, c, cl, *mat)
        rho, u = inputs(m, 60 + k)
        rho[::5] = 1e-9
        rho[1::7] = 0.0
        meshes.append(m)
        rhos.append(to_dev(rho))
        us.append(to_dev(u))
    got = step_group(meshes, rhos, us)
    for m, rho, u, (vals, dc, cc) in zip(meshes, rhos, us, got):
        v1, d1, c1 = m.step(rho, u)
        assert torch.equal(vals, v1) and torch.equal(dc, d1) and torch.equal(cc, c1)


def test_group_arguments(lib):
    import ctypes
    from paper_2505_02438_gb300 import _native as N
    from paper_2505_02438_gb300 import step_group
    c, cl = W.structured_quad(6, 4)
    m = lib.Mesh("quad", 1, c, cl, *MAT)
    rho, u = inputs(m, 1)
    with pytest.raises(N.SoptxError) as ei:
        step_group([m, m], [to_dev(rho)] * 2, [to_dev(u)] * 2)
    assert ei.value.code == 1
    assert step_group([], [], []) == []
    P = ctypes.c_void_p * 1
    assert N.lib().soptx_assemble_and_sensitivity_group(1, P(m._h.value), P(None), P(None), P(None), P(None),
                                                        P(None), None) == 1
