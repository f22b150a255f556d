"""Python handle on the steps after the sensitivities (include/soptx_opt.h):
the sensitivity / density filters, the Heaviside projection and the
optimality-criteria update, and the optimisation loop that chains them with
the assembly, the constrained solve and the sensitivities.  Argument
marshalling and loop control only: every step runs in the library."""
import ctypes

import numpy as np
import torch

from . import _native as N
from .api import _dptr, _stream


def cell_centroids_volumes(cell, coords, cells):
    """Centroids (mean of the vertices) and volumes of the cells of a mesh:
    simplices |det J| / d!, tensor cells by the 2-point Gauss rule of their
    multilinear map (exact for bilinear / trilinear cells)."""
    coords = np.asarray(coords, np.float64)
    cells = np.asarray(cells, np.int64)
    xv = coords[cells]                     # [nc, nv, d]
    cen = xv.mean(axis=1)
    d = coords.shape[1]
    if cell in ("tri", "tet"):
        J = xv[:, 1:, :] - xv[:, :1, :]
        return cen, np.abs(np.linalg.det(J)) / (2.0 if d == 2 else 6.0)
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    vol = np.zeros(len(cells))
    nvc = 1 << d
    for pt in np.stack(np.meshgrid(*([g] * d), indexing="ij"), -1).reshape(-1, d):
        dN = np.zeros((nvc, d))
        for v in range(nvc):
            for m in range(d):
                s = 1.0 if (v >> m) & 1 else -1.0
                for o in range(d):
                    if o != m:
                        s *= pt[o] if (v >> o) & 1 else 1.0 - pt[o]
                dN[v, m] = s
        vol += np.abs(np.linalg.det(np.einsum("evi,vm->eim", xv, dN))) / (2 ** d)
    return cen, vol


class Filter:
    """H_ij = max(0, rmin - |c_i - c_j|) over the cells' centroids, on the device."""

    def __init__(self, centroids, volumes, rmin, device=None):
        cen = np.ascontiguousarray(centroids, np.float64)
        vol = np.ascontiguousarray(volumes, np.float64)
        self.n, self.dim = cen.shape
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        h = ctypes.c_void_p()
        N.check(N.lib().soptx_filter_create(self.dim, self.n, cen.ctypes.data_as(ctypes.c_void_p),
                                            vol.ctypes.data_as(ctypes.c_void_p), float(rmin), _stream(None),
                                            ctypes.byref(h)))
        self._h = h
        nc, nnz = ctypes.c_int64(), ctypes.c_int64()
        N.check(N.lib().soptx_filter_info(h, ctypes.byref(nc), ctypes.byref(nnz)))
        self.nnz = nnz.value

    def _out(self, out):
        return torch.empty(self.n, dtype=torch.float64, device=self.device) if out is None else out

    def sensitivity(self, rho, dc, out=None):
        out = self._out(out)
        N.check(N.lib().soptx_filter_sensitivity(self._h, _dptr(rho, torch.float64, self.n, "rho"),
                                                 _dptr(dc, torch.float64, self.n, "dc"),
                                                 _dptr(out, torch.float64, self.n, "out"), _stream(None)))
        return out

    def density(self, x, out=None):
        out = self._out(out)
        N.check(N.lib().soptx_filter_density(self._h, _dptr(x, torch.float64, self.n, "x"),
                                             _dptr(out, torch.float64, self.n, "out"), _stream(None)))
        return out

    def density_grad(self, g, out=None):
        out = self._out(out)
        N.check(N.lib().soptx_filter_density_grad(self._h, _dptr(g, torch.float64, self.n, "g"),
                                                  _dptr(out, torch.float64, self.n, "out"), _stream(None)))
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib().soptx_filter_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def heaviside(x, beta, want_derivative=False):
    n = x.numel()
    out = torch.empty_like(x)
    dout = torch.empty_like(x) if want_derivative else None
    N.check(N.lib().soptx_heaviside(n, float(beta), _dptr(x, torch.float64, n, "x"),
                                    _dptr(out, torch.float64, n, "out"),
                                    _dptr(dout, torch.float64, n, "dout") if want_derivative else None,
                                    _stream(None)))
    return (out, dout) if want_derivative else out


def oc_update(rho, dc, dv, vol, volfrac, move=0.2, eta=0.5, l_lo=0.0, l_hi=1e9, tol=1e-3):
    """Optimality-criteria update; returns (rho_new, dict(change, lam, vol_frac))."""
    n = rho.numel()
    out = torch.empty_like(rho)
    stats = torch.empty(3, dtype=torch.float64, device=rho.device)
    o = N.OcOpts(float(volfrac), float(move), float(eta), float(l_lo), float(l_hi), float(tol))
    N.check(N.lib().soptx_oc_update(n, _dptr(rho, torch.float64, n, "rho"), _dptr(dc, torch.float64, n, "dc"),
                                    _dptr(dv, torch.float64, n, "dv"), _dptr(vol, torch.float64, n, "vol"),
                                    ctypes.byref(o), _dptr(out, torch.float64, n, "out"),
                                    _dptr(stats, torch.float64, 3, "stats"), _stream(None)))
    st = stats.cpu().numpy()
    return out, dict(change=float(st[0]), lam=float(st[1]), vol_frac=float(st[2]))


def oc_loop(mesh, fixed, f, rmin, volfrac, vol, centroids, max_iter=200, tol=1e-2, move=0.2, eta=0.5,
            cg_rtol=1e-10, cg_max_iter=200000, callback=None):
    """Compliance minimisation with the sensitivity filter and the OC update
    (Algorithm 1), every step on the device: K(rho) assembly, the constrained
    CG solve (warm-started from the previous design's displacements), the
    sensitivities, the filter and the update, until max |rho_new - rho| <= tol.
    Returns dict(rho, u, history=[(c, volume fraction, change, CG iterations)])."""
    dev = mesh.device
    flt = Filter(centroids, vol, rmin)
    vol_t = torch.as_tensor(np.asarray(vol, np.float64), device=dev)
    fixed_t = torch.as_tensor(np.asarray(fixed), device=dev).to(torch.uint8)
    f_t = torch.as_tensor(np.asarray(f, np.float64), device=dev)
    x = torch.full((mesh.n_cells,), float(volfrac), dtype=torch.float64, device=dev)
    u = None
    hist = []
    for it in range(max_iter):
        vals = mesh.assemble_K(x)
        u, info = mesh.solve(vals, fixed_t, f_t, rtol=cg_rtol, max_iter=cg_max_iter, check_every=50, u0=u)
        dc, c = mesh.sensitivity(x, u)
        dcf = flt.sensitivity(x, dc)
        xnew, st = oc_update(x, dcf, vol_t, vol_t, volfrac, move=move, eta=eta)
        hist.append((c.item(), st["vol_frac"], st["change"], info["iterations"]))
        if callback:
            callback(it, hist[-1])
        x = xnew
        if st["change"] <= tol:
            break
    flt.close()
    return dict(rho=x, u=u, history=hist)
