"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle,
element by element, on every cell type and order (several tiles and ragged
tails per kernel), both element precisions, and the edge cases."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from helpers import TOL32, TOL64, oracle_csr, small_cases
from paper_2505_02438_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MAT = (1.0, 1e-9, 0.3, 3.0, 0)
CASES = small_cases()


@pytest.fixture(scope="module")
def P(lib):
    assert torch.cuda.is_available()
    return lib


def to_dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def check_assembly(P, cell, k, coords, cells, prec, mat=MAT, seed=0):
    m = P.Mesh(cell, k, coords, cells, *mat, elem_prec=prec)
    g = np.random.default_rng(seed)
    rho = g.uniform(0.001, 1.0, len(cells))
    vals = m.assemble_K(to_dev(rho))
    indptr, indices = m.pattern()
    rp, ci, v, va, ndof = oracle_csr(cell, k, coords, cells, mat, rho)
    assert m.ndof == ndof and m.nnz == len(v)
    assert np.array_equal(indptr.cpu().numpy(), rp)
    assert np.array_equal(indices.cpu().numpy(), ci)
    got = vals.cpu().numpy()
    err = np.abs(got - v)
    tol = TOL64 if prec == "fp64" else TOL32
    floor = (1e-15 if prec == "fp64" else 1e-7) * va.max(initial=0.0)
    bad = err > tol * va + floor
    assert not bad.any(), (prec, np.argmax(err / (va + 1e-300)), (err / (va + floor + 1e-300)).max())
    u = g.standard_normal(ndof)
    dc, c = m.sensitivity(to_dev(rho), to_dev(u))
    dco, so, co, sabs = oracle.sensitivity(cell, k, coords, cells, mat, rho, u, with_abs=True)
    E0, Emin, nu, p, ps = mat
    dE = p * rho ** (p - 1) * (E0 - Emin)
    E = Emin + rho ** p * (E0 - Emin)
    dcg = dc.cpu().numpy()
    assert np.all(np.abs(dcg - dco) <= tol * dE * sabs + 1e-300), np.max(np.abs(dcg - dco) / (dE * sabs))
    assert abs(c.item() - co) <= tol * np.dot(E, sabs)
    return m, rho, u, vals, dc, c, (err / (va + floor + 1e-300)).max()


@pytest.mark.parametrize("name,cell,k,coords,cells", CASES, ids=[c[0] for c in CASES])
def test_fp64_matches_oracle(P, name, cell, k, coords, cells):
    m, rho, u, vals, dc, c, _ = check_assembly(P, cell, k, coords, cells, "fp64")
    expected_path = "lattice" if "lattice" in name else (
        "uniform" if cell in ("quad", "hex") and "distorted" not in name else "cached")
    assert m.path == expected_path
    # the fused step gives the same bits as the separate calls, and reruns are bitwise equal
    v2, dc2, c2 = m.step(to_dev(rho), to_dev(u))
    assert torch.equal(v2, vals) and torch.equal(dc2, dc) and torch.equal(c2, c)
    v3 = m.assemble_K(to_dev(rho))
    assert torch.equal(v3, vals)


@pytest.mark.parametrize("name,cell,k,coords,cells", [c for c in CASES if c[2] <= 2 or c[1] == "tri"],
                         ids=[c[0] for c in CASES if c[2] <= 2 or c[1] == "tri"])
def test_fp32_elements_match_oracle(P, name, cell, k, coords, cells):
    check_assembly(P, cell, k, coords, cells, "fp32")


@pytest.mark.parametrize("mat", [(1.0, 0.0, 0.3, 3.0, 0), (2.5, 1e-6, 0.25, 2.5, 1), (1.0, 1e-9, 0.0, 1.0, 0)])
def test_material_variants(P, mat):
    c, cl = W.triangle_grid(9, 5, 0.2, np.random.default_rng(3))
    check_assembly(P, "tri", 2, c, cl, "fp64", mat=mat)
    c, cl = W.structured_quad(9, 4)
    check_assembly(P, "quad", 1, c, cl, "fp64", mat=mat)
    c, cl = W.structured_hex(3, 3, 2)
    check_assembly(P, "hex", 1, c, cl, "fp64", mat=(mat[0], mat[1], mat[2], mat[3], 0))


def test_single_element_and_extreme_densities(P):
    for cell, k, (c, cl) in [("hex", 1, W.structured_hex(1, 1, 1)), ("tet", 3, W.kuhn_tets(1, 1, 1)),
                             ("quad", 1, W.structured_quad(1, 1)), ("tri", 3, W.triangle_grid(1, 1))]:
        cl1 = cl[:1]
        used = np.unique(cl1)
        remap = -np.ones(len(c), np.int64)
        remap[used] = np.arange(len(used))
        check_assembly(P, cell, k, c[used], remap[cl1].astype(np.int32), "fp64")
    c, cl = W.structured_hex(5, 4, 3)
    m = P.Mesh("hex", 1, c, cl)
    for r in (np.full(len(cl), 0.001), np.ones(len(cl)), np.where(np.arange(len(cl)) % 2, 1.0, 0.001)):
        vals = m.assemble_K(to_dev(r)).cpu().numpy()
        rp, ci, v, va, _ = oracle_csr("hex", 1, c, cl, MAT, r)
        assert np.all(np.abs(vals - v) <= TOL64 * va + 1e-15 * va.max())


def test_empty_mesh(P):
    m = P.Mesh("tri", 2, np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]), np.zeros((0, 3), np.int32))
    assert m.ndof == 6 and m.nnz == 0 and m.n_cells == 0
    rho = torch.zeros(0, dtype=torch.float64, device="cuda")
    vals = m.assemble_K(rho)
    dc, c = m.sensitivity(rho, torch.zeros(6, dtype=torch.float64, device="cuda"))
    assert vals.numel() == 0 and dc.numel() == 0 and c.item() == 0.0
    gr, gu = m.compliance_vjp(rho, torch.ones(6, dtype=torch.float64, device="cuda"),
                              torch.ones(1, dtype=torch.float64, device="cuda"))
    assert gr.numel() == 0 and torch.equal(gu.cpu(), torch.zeros(6, dtype=torch.float64))


def test_invalid_arguments_raise(P):
    from paper_2505_02438_gb300 import _native as N
    c, cl = W.structured_quad(3, 3)
    m = P.Mesh("quad", 1, c, cl)
    with pytest.raises(TypeError):
        m.assemble_K(torch.zeros(m.n_cells, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        m.assemble_K(torch.zeros(m.n_cells + 1, dtype=torch.float64, device="cuda"))
    with pytest.raises(N.SoptxError):
        P.Mesh("quad", 1, c, cl, nu=0.5)
    with pytest.raises(N.SoptxError):
        P.Mesh("quad", 1, c, cl, E0=1.0, Emin=2.0)


def test_allocation_failure_rolls_back(P):
    from paper_2505_02438_gb300 import _native as N
    c, cl = W.kuhn_tets(3, 2, 2, 0.1, np.random.default_rng(0))
    for n in (1, 3, 7, 11):
        N.lib().soptx_debug_fail_alloc_after(n)
        try:
            with pytest.raises(N.SoptxError) as ei:
                P.Mesh("tet", 2, c, cl)
            assert ei.value.code == 2
        finally:
            N.lib().soptx_debug_fail_alloc_after(0)
    m = P.Mesh("tet", 2, c, cl)          # the library is still usable
    assert m.nnz > 0


@pytest.mark.parametrize("cell,mk", [("hex", lambda: W.structured_hex(5, 4, 3)), ("quad", lambda: W.structured_quad(9, 7))])
def test_lattice_out_of_range_moduli_take_fp64_route(P, cell, mk):
    """With Emin = 0, tiny densities give moduli below the float-pair range;
    those nodes are assembled in plain FP64 and must still match."""
    c, cl = mk()
    mat = (1.0, 0.0, 0.3, 3.0, 0)
    m = P.Mesh(cell, 1, c, cl, *mat)
    assert m.path == "lattice"
    g = np.random.default_rng(8)
    rho = g.uniform(0.001, 1.0, len(cl))
    rho[::5] = 1e-9          # E = 1e-27
    rho[1::7] = 0.0          # E = 0 exactly
    vals = m.assemble_K(to_dev(rho)).cpu().numpy()
    rp, ci, v, va, _ = oracle_csr(cell, 1, c, cl, mat, rho)
    assert np.all(np.abs(vals - v) <= TOL64 * va + 1e-300)


GENERAL_OOR = [c for c in CASES if c[0] in ("tet_p2_5x3x2_jitter", "tri_p3_17x9_jitter", "hex_q1_relabelled_uniform",
                                           "quad_q1_9x6_distorted", "hex_q1_5x4x3_distorted", "tet_p1_5x3x2_jitter",
                                           "quad_q2_7x5")]


@pytest.mark.parametrize("name,cell,k,coords,cells", GENERAL_OOR, ids=[c[0] for c in GENERAL_OOR])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_general_out_of_range_moduli_take_fp64_route(P, name, cell, k, coords, cells, prec):
    """The general gathers (every row layout, with and without the
    sensitivity, and the generic node gather) with moduli below the
    float-pair range: those nodes are gathered in plain FP64, the results match
    the oracle, and the one-call step gives the bits of the separate calls."""
    mat = (1.0, 0.0, 0.3, 3.0, 0)
    m = P.Mesh(cell, k, coords, cells, *mat, elem_prec=prec)
    assert m.path in ("cached", "uniform")
    g = np.random.default_rng(12)
    rho = g.uniform(0.001, 1.0, len(cells))
    rho[::5] = 1e-9          # E = 1e-27
    rho[1::7] = 0.0          # E = 0 exactly
    rho[3::11] = 1e-30       # E = 1e-90
    vals = m.assemble_K(to_dev(rho))
    rp, ci, v, va, ndof = oracle_csr(cell, k, coords, cells, mat, rho)
    tol = TOL64 if prec == "fp64" else TOL32
    err = np.abs(vals.cpu().numpy() - v)
    # entries that vanish in exact arithmetic carry rounding noise in both codes: an absolute floor
    # relative to the largest entry and, for the entries whose node pair shares tiny cells only (the
    # FP64 route this test is about), relative to the largest of those
    assert np.all(err <= tol * va + (1e-15 if prec == "fp64" else 1e-7) * va.max() + 1e-300)
    cn, nn = oracle.number(cell, k, len(coords), cells)
    d = 2 if cell in ("tri", "quad") else 3
    pairs = lambda sel: sp.coo_matrix((np.ones(sel.sum() * cn.shape[1] ** 2),
                                       (np.repeat(cn[sel], cn.shape[1], axis=1).ravel(),
                                        np.tile(cn[sel], (1, cn.shape[1])).ravel())), shape=(nn, nn)).tocsr()
    normal, small = pairs(rho >= 1e-8), pairs((rho < 1e-8) & (rho > 0))
    row = np.repeat(np.arange(len(rp) - 1), np.diff(rp)) // d
    col = ci // d
    tiny = (np.asarray(small[row, col]).ravel() > 0) & (np.asarray(normal[row, col]).ravel() == 0)
    assert tiny.any()
    fl = 1e-15 if prec == "fp64" else 1e-6
    assert np.all(err[tiny] <= tol * va[tiny] + fl * va[tiny].max() + 1e-300)
    u = g.standard_normal(ndof)
    dc, c = m.sensitivity(to_dev(rho), to_dev(u))
    dco, so, co, sabs = oracle.sensitivity(cell, k, coords, cells, mat, rho, u, with_abs=True)
    dE = 3.0 * rho ** 2
    assert np.all(np.abs(dc.cpu().numpy() - dco) <= tol * dE * sabs + 1e-300)
    v2, dc2, c2 = m.step(to_dev(rho), to_dev(u))
    assert torch.equal(v2, vals) and torch.equal(dc2, dc) and torch.equal(c2, c)


def test_lattice_out_of_range_moduli_between_normal_calls(P):
    """Calls with and without out-of-range moduli alternate on one 3D lattice
    (several warps and blocks, cells of both kinds next to chunk borders): each
    call matches the oracle, so no state of one call leaks into the next."""
    c, cl = W.structured_hex(23, 9, 7)
    mat = (1.0, 0.0, 0.3, 3.0, 0)
    m = P.Mesh("hex", 1, c, cl, *mat)
    assert m.path == "lattice"
    g = np.random.default_rng(9)
    normal = g.uniform(0.001, 1.0, len(cl))
    tiny = normal.copy()
    tiny[g.choice(len(cl), 40, replace=False)] = 1e-9      # E = 1e-27
    tiny[g.choice(len(cl), 10, replace=False)] = 1e-30     # E = 1e-90, below the float range
    for rho in (normal, tiny, normal, tiny, tiny, normal):
        vals = m.assemble_K(to_dev(rho)).cpu().numpy()
        rp, ci, v, va, _ = oracle_csr("hex", 1, c, cl, mat, rho)
        assert np.all(np.abs(vals - v) <= TOL64 * va + 1e-300)


def test_extreme_box_aspect_takes_general_path(P):
    """Boxes whose element matrix entries span more than 2^24 (aspect ratio
    10^4) leave the lattice kernels for the general path, and still match."""
    c, cl = W.structured_hex(4, 3, 3)
    c = c * np.array([1.0, 1.0, 1e-4])
    m, *_ = check_assembly(P, "hex", 1, c, cl, "fp64")
    assert m.path == "uniform"


@pytest.mark.parametrize("n", [(2, 2, 2), (4, 2, 2), (4, 4, 2), (16, 3, 2)])
def test_lattice_node_pairs_with_odd_tails(P, n):
    """The 3D lattice assembly takes two nodes per pass within chunks of 16:
    node counts 27, 45 and 75 leave a lone node at the end, and with an odd
    number of nodes per row (3, 5, 17) some pairs straddle two rows."""
    c, cl = W.structured_hex(*n)
    m, *_ = check_assembly(P, "hex", 1, c, cl, "fp64", seed=11)
    assert m.path == "lattice"


def test_lattice_anisotropic_boxes(P):
    """Box cells with different edge lengths per axis and a shifted origin."""
    c, cl = W.structured_hex(6, 4, 3)
    c = c * np.array([0.5, 1.25, 2.0]) + np.array([3.0, -1.0, 0.25])
    m, *_ = check_assembly(P, "hex", 1, c, cl, "fp64")
    assert m.path == "lattice"
    c, cl = W.structured_quad(8, 5)
    c = c * np.array([2.0, 0.3])
    m, *_ = check_assembly(P, "quad", 1, c, cl, "fp64")
    assert m.path == "lattice"


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("cell,mk", [("hex", lambda: W.structured_hex(6, 5, 4)), ("quad", lambda: W.structured_quad(11, 7))])
def test_lattice_without_sectors_uses_general_sensitivity(P, cell, mk, prec):
    """A box lattice whose element matrix is not split into Walsh sectors
    computes its sensitivities with the general gather kernels."""
    from paper_2505_02438_gb300 import _native as N
    coords, cells = mk()
    N.lib().soptx_debug_lattice_no_sectors(1)
    try:
        m, *_ = check_assembly(P, cell, 1, coords, cells, prec)
    finally:
        N.lib().soptx_debug_lattice_no_sectors(0)
    assert m.path == "lattice"


HOST_CASES = [c for c in CASES if c[0] in ("hex_q1_13x5x4_lattice", "q4_60x20_lattice", "tet_p2_5x3x2_jitter",
                                           "hex_q1_relabelled_uniform")]


@pytest.mark.parametrize("name,cell,k,coords,cells", HOST_CASES, ids=[c[0] for c in HOST_CASES])
def test_step_host_matches_device_step(P, name, cell, k, coords, cells):
    """soptx_step_host (host rho, u, dc, c; on a box lattice the sensitivities
    on a second stream) gives the bits of the device-pointer step, call after
    call with changing inputs, with dc and c in one buffer or two, c omitted,
    and pageable host memory."""
    import ctypes
    from paper_2505_02438_gb300 import _native as N
    m = P.Mesh(cell, k, coords, cells)
    g = np.random.default_rng(21)
    for it in range(3):
        rho = g.uniform(0.001, 1.0, len(cells))
        u = g.standard_normal(m.ndof)
        v_ref, dc_ref, c_ref = m.step(to_dev(rho), to_dev(u))
        torch.cuda.synchronize()
        pin = it != 2
        rho_h = torch.as_tensor(rho).pin_memory() if pin else torch.as_tensor(rho).clone()
        u_h = torch.as_tensor(u).pin_memory() if pin else torch.as_tensor(u).clone()
        vals, dc_h, c_h = m.step_host(rho_h, u_h)
        torch.cuda.synchronize()
        assert torch.equal(vals, v_ref)
        assert torch.equal(dc_h, dc_ref.cpu()) and torch.equal(c_h, c_ref.cpu())
    # dc and c in separate buffers, then without c
    dc2 = torch.full((m.n_cells,), np.nan, dtype=torch.float64).pin_memory()
    c2 = torch.full((1,), np.nan, dtype=torch.float64).pin_memory()
    vals2 = torch.empty_like(v_ref)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for cptr in (ctypes.c_void_p(c2.data_ptr()), None):
        N.check(N.lib().soptx_step_host(m._h, ctypes.c_void_p(rho_h.data_ptr()), ctypes.c_void_p(u_h.data_ptr()),
                                        ctypes.c_void_p(vals2.data_ptr()), ctypes.c_void_p(dc2.data_ptr()), cptr, st))
        torch.cuda.synchronize()
        assert torch.equal(vals2, v_ref) and torch.equal(dc2, dc_ref.cpu()) and torch.equal(c2, c_ref.cpu())
    with pytest.raises(N.SoptxError):
        N.check(N.lib().soptx_step_host(m._h, None, ctypes.c_void_p(u_h.data_ptr()),
                                        ctypes.c_void_p(vals2.data_ptr()), ctypes.c_void_p(dc2.data_ptr()), None, st))


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_hex_sensitivities_by_sum_factorisation(P, k, prec):
    """Hexahedra of order 2 and 3 take the sum-factorised strain-energy kernel:
    a sheared box (parallelepipeds, so G is a full matrix) against the oracle,
    both element precisions."""
    c, cl = W.structured_hex(3, 2, 2)
    shear = np.array([[1.0, 0.3, -0.2], [0.1, 0.9, 0.25], [-0.15, 0.2, 1.1]])
    coords = c @ shear.T + np.array([0.5, -1.0, 2.0])
    m = P.Mesh("hex", k, coords, cl, *MAT, elem_prec=prec)
    assert m.routes["sensitivity"] == "strain"
    g = np.random.default_rng(20 + k)
    rho = g.uniform(0.001, 1.0, len(cl))
    u = g.standard_normal(m.ndof)
    dc, cc = m.sensitivity(to_dev(rho), to_dev(u))
    dco, so, co, sabs = oracle.sensitivity("hex", k, coords, cl, MAT, rho, u, with_abs=True)
    E0, Emin, nu, p, ps = MAT
    dE = p * rho ** (p - 1) * (E0 - Emin)
    E = Emin + rho ** p * (E0 - Emin)
    tol = TOL64 if prec == "fp64" else TOL32
    assert np.all(np.abs(dc.cpu().numpy() - dco) <= tol * dE * sabs + 1e-300)
    assert abs(cc.item() - co) <= tol * np.dot(E, sabs)
