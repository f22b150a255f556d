"""The differentiation pattern: Compliance.apply forward/backward against the
oracle's gradient and central finite differences (step 1e-6)."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL64
from paper_2505_02438_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def fd_tolerance(E0, Emin, s, h, f, grad):
    """f is cubic in rho_e (p = 3): the central-difference truncation error is
    exactly (E0 - Emin) s_e h^2; rounding adds about 4 eps |f| / h."""
    return (E0 - Emin) * np.abs(s) * h * h + 8 * np.finfo(float).eps * abs(f) / h + 1e-8 * np.abs(grad)


@pytest.mark.parametrize("mk", [lambda: W.jittered_tet(5, 3, 2, order=2), lambda: W.cantilever_hex(6, 4, 3),
                                lambda: W.jittered_tri(9, 6, order=3)])
def test_compliance_backward_matches_oracle_and_fd(lib, mk):
    from paper_2505_02438_gb300.autograd import Compliance
    wl = mk()
    m = lib.Mesh.from_workload(wl)
    u_np = wl.displacement(m.ndof)
    rho = torch.as_tensor(wl.rho, device="cuda").requires_grad_(True)
    u = torch.as_tensor(u_np, device="cuda").requires_grad_(True)
    c = Compliance.apply(rho, u, m)
    assert c.dim() == 0
    (2.5 * c).backward()
    g = 2.5
    gr_o, gu_o = oracle.compliance_vjp(wl.cell, wl.order, wl.coords, wl.cells, wl.mat, wl.rho, u_np, g)
    dco, s, co, sabs = oracle.sensitivity(wl.cell, wl.order, wl.coords, wl.cells, wl.mat, wl.rho, u_np, with_abs=True)
    E0, Emin, nu, p, ps = wl.mat
    dE = p * wl.rho ** (p - 1) * (E0 - Emin)
    E = Emin + wl.rho ** p * (E0 - Emin)
    assert abs(c.item() - co) <= TOL64 * np.dot(E, sabs)
    gr = rho.grad.cpu().numpy()
    assert np.all(np.abs(gr - gr_o) <= TOL64 * g * dE * sabs)
    # u-gradient 2 g K u: scale = 2 g |K| |u|
    rp, ci, va, _ = oracle.assemble(wl.cell, wl.order, wl.coords, wl.cells, wl.mat, wl.rho, absval=True)
    scale = np.array([np.dot(va[rp[r]:rp[r + 1]], np.abs(u_np[ci[rp[r]:rp[r + 1]]])) for r in range(m.ndof)])
    gu = u.grad.cpu().numpy()
    assert np.all(np.abs(gu - gu_o) <= TOL64 * 2 * g * scale)
    # central differences of the GPU forward in rho
    h = 1e-6
    idx = np.random.default_rng(0).choice(len(wl.cells), size=min(16, len(wl.cells)), replace=False)
    with torch.no_grad():
        for e in idx:
            rp_ = torch.as_tensor(wl.rho, device="cuda").clone()
            rm_ = rp_.clone()
            rp_[e] += h
            rm_[e] -= h
            fd = g * (Compliance.apply(rp_, u, m).item() - Compliance.apply(rm_, u, m).item()) / (2 * h)
            assert abs(fd - gr[e]) <= g * fd_tolerance(E0, Emin, s[e], h, co, gr[e] / g), (e, fd, gr[e])


def test_grad_only_rho(lib):
    from paper_2505_02438_gb300.autograd import Compliance
    wl = W.jittered_tet(3, 2, 2, order=2)
    m = lib.Mesh.from_workload(wl)
    rho = torch.as_tensor(wl.rho, device="cuda").requires_grad_(True)
    u = torch.as_tensor(wl.displacement(m.ndof), device="cuda")
    Compliance.apply(rho, u, m).backward()
    dc, _ = m.sensitivity(rho.detach(), u)
    # rho-gradient of u^T K(rho) u is minus the compliance sensitivity, bit for bit on this path
    assert torch.allclose(rho.grad, -dc, rtol=1e-14, atol=0)


@pytest.mark.parametrize("mk", [lambda: W.cantilever_hex(6, 4, 3), lambda: W.jittered_tet(4, 3, 2, order=2)])
def test_u_gradient_assembled_and_matrix_free(lib, mk):
    """The u-gradient 2 g K(rho) u goes through K(rho) assembled into the mesh's
    scratch; when that scratch cannot be allocated it is formed matrix-free.
    Both match the oracle."""
    import ctypes
    from paper_2505_02438_gb300 import _native as N
    wl = mk()
    g = 1.75
    gr_o, gu_o = oracle.compliance_vjp(wl.cell, wl.order, wl.coords, wl.cells, wl.mat, wl.rho,
                                       wl.displacement(lib.Mesh.from_workload(wl).ndof), g)
    rp, ci, va, _ = oracle.assemble(wl.cell, wl.order, wl.coords, wl.cells, wl.mat, wl.rho, absval=True)
    for fail in (1, 0):
        m = lib.Mesh.from_workload(wl)
        u_np = wl.displacement(m.ndof)
        scale = np.array([np.dot(va[rp[r]:rp[r + 1]], np.abs(u_np[ci[rp[r]:rp[r + 1]]])) for r in range(m.ndof)])
        try:
            N.lib().soptx_debug_fail_alloc_after(fail)
            gr, gu = m.compliance_vjp(torch.as_tensor(wl.rho, device="cuda"), torch.as_tensor(u_np, device="cuda"),
                                      torch.tensor([g], dtype=torch.float64, device="cuda"))
        finally:
            N.lib().soptx_debug_fail_alloc_after(0)
        torch.cuda.synchronize()
        nbytes = ctypes.c_int64(0)
        N.check(N.lib().soptx_mesh_device_bytes(m._h, ctypes.byref(nbytes)))
        assert nbytes.value == m.device_bytes + (0 if fail else 8 * m.nnz)   # the scratch only when it was had
        assert np.all(np.abs(gu.cpu().numpy() - gu_o) <= TOL64 * 2 * g * scale)
        dco, s, co, sabs = oracle.sensitivity(wl.cell, wl.order, wl.coords, wl.cells, wl.mat, wl.rho, u_np,
                                              with_abs=True)
        E0, Emin, nu, p, ps = wl.mat
        assert np.all(np.abs(gr.cpu().numpy() - gr_o) <= TOL64 * g * p * wl.rho ** (p - 1) * (E0 - Emin) * sabs)
