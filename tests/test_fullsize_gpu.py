"""Parity at the full workload sizes, in the launch configuration the benchmark
times: the whole pattern's structure, sampled CSR rows and sampled cells
against the oracle (which computes them one by one), and properties that hold
at any size."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL32, TOL64
from paper_2505_02438_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FULL = {
    "hex": lambda: W.cantilever_hex(120, 40, 40),
    "tri": lambda: W.jittered_tri(400, 200),
    "tet": lambda: W.jittered_tet(60, 20, 20),
}


def run_full(lib, name, prec="fp64"):
    wl = FULL[name]()
    m = lib.Mesh.from_workload(wl, elem_prec=prec)
    rho = torch.as_tensor(wl.rho, device="cuda")
    u_np = wl.displacement(m.ndof)
    u = torch.as_tensor(u_np, device="cuda")
    vals, dc, c = m.step(rho, u)
    indptr, indices = m.pattern()
    torch.cuda.synchronize()
    return wl, m, u_np, vals.cpu().numpy(), dc.cpu().numpy(), c.item(), indptr.cpu().numpy(), indices.cpu().numpy()


@pytest.mark.parametrize("name,prec", [("hex", "fp64"), ("tri", "fp64"), ("tet", "fp64"), ("tri", "fp32")])
def test_full_size_sampled_parity(lib, name, prec):
    wl, m, u_np, vals, dc, c, indptr, indices = run_full(lib, name, prec)
    d = wl.dim
    # structure at any size: rows sorted and unique, the d rows of a node identical in columns
    assert indptr[0] == 0 and indptr[-1] == m.nnz and np.all(np.diff(indptr) > 0)
    g = np.random.default_rng(77)
    rows = np.unique(np.concatenate([[0, m.ndof - 1], g.choice(m.ndof, 400, replace=False)]))
    for r in rows[:50]:
        cols = indices[indptr[r]:indptr[r + 1]]
        assert np.all(np.diff(cols) > 0)
    rp, ci, v, ndof = oracle.assemble(wl.cell, wl.order, wl.coords, wl.cells, wl.mat, wl.rho, rows=rows)
    _, _, va, _ = oracle.assemble(wl.cell, wl.order, wl.coords, wl.cells, wl.mat, wl.rho, rows=rows, absval=True)
    assert ndof == m.ndof
    tol = TOL64 if prec == "fp64" else TOL32
    worst = 0.0
    rel = []
    for s, r in enumerate(rows):
        sl = slice(indptr[r], indptr[r + 1])
        assert np.array_equal(indices[sl], ci[rp[s]:rp[s + 1]]), r
        err = np.abs(vals[sl] - v[rp[s]:rp[s + 1]])
        scale = va[rp[s]:rp[s + 1]]
        floor = (1e-15 if prec == "fp64" else 1e-7) * scale.max()
        assert np.all(err <= tol * scale + floor), r
        # error relative to the entry's scale (sum of |contributions|, plus the row floor)
        rel.append(err / (scale + floor / tol))
        worst = max(worst, float(rel[-1].max()))
    rel = np.concatenate(rel)
    print("%s %s: sampled rows %d, max rel err %.3e, rms %.3e" % (name, prec, len(rows), worst, np.sqrt(np.mean(rel ** 2))))
    cells = np.unique(np.concatenate([[0, len(wl.cells) - 1], g.choice(len(wl.cells), 300, replace=False)]))
    dco, so, _, sabs = oracle.sensitivity(wl.cell, wl.order, wl.coords, wl.cells, wl.mat, wl.rho, u_np, sel=cells,
                                          with_abs=True)
    E0, Emin, nu, p, ps = wl.mat
    r_ = wl.rho[cells]
    dE = p * r_ ** (p - 1) * (E0 - Emin)
    assert np.all(np.abs(dc[cells] - dco) <= tol * dE * sabs)
    # c is the sum of E_e s_e with s_e = -dc_e / E'_e (a property at any size)
    dE_all = p * wl.rho ** (p - 1) * (E0 - Emin)
    E_all = Emin + wl.rho ** p * (E0 - Emin)
    s_all = -dc / dE_all
    assert abs(c - np.dot(E_all, s_all)) <= 1e-10 * np.dot(E_all, np.abs(s_all))


def test_full_size_tet_fd_64_cells(lib):
    """Kuhn P2 tets at full size: Compliance backward against central
    differences (step 1e-6) on 64 seeded cells."""
    from paper_2505_02438_gb300.autograd import Compliance
    wl = FULL["tet"]()
    m = lib.Mesh.from_workload(wl)
    u = torch.as_tensor(wl.displacement(m.ndof), device="cuda")
    rho = torch.as_tensor(wl.rho, device="cuda").requires_grad_(True)
    f = Compliance.apply(rho, u, m)
    f.backward()
    grad = rho.grad.cpu().numpy()
    dc, _ = m.sensitivity(rho.detach(), u)
    s = -dc.cpu().numpy() / (wl.p * wl.rho ** (wl.p - 1) * (wl.E0 - wl.Emin))
    h = 1e-6
    cells = np.random.default_rng(4).choice(len(wl.cells), 64, replace=False)
    with torch.no_grad():
        for e in cells:
            rp_ = rho.detach().clone()
            rm_ = rp_.clone()
            rp_[e] += h
            rm_[e] -= h
            fd = (Compliance.apply(rp_, u, m).item() - Compliance.apply(rm_, u, m).item()) / (2 * h)
            tol = (wl.E0 - wl.Emin) * abs(s[e]) * h * h + 8 * np.finfo(float).eps * abs(f.item()) / h + 1e-8 * abs(grad[e])
            assert abs(fd - grad[e]) <= tol, (e, fd, grad[e], tol)
