"""Python binding of the SIMP assembly library: torch tensors in, torch tensors out.

Each method marshals its arguments (device pointers of contiguous CUDA float64
tensors, the current CUDA stream) and calls the C ABI; every step of the path
runs in the library's kernels.
"""
import ctypes

import numpy as np
import torch

from . import _native as N


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t, dtype, n, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError("%s must be contiguous with %d elements (got %s)" % (name, n, tuple(t.shape)))
    return ctypes.c_void_p(t.data_ptr())


def _hptr(t, n, name):
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("%s must be a host (CPU) tensor" % name)
    if t.dtype != torch.float64:
        raise TypeError("%s must have dtype torch.float64, got %s" % (name, t.dtype))
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError("%s must be contiguous with %d elements (got %s)" % (name, n, tuple(t.shape)))
    return ctypes.c_void_p(t.data_ptr())


class Mesh:
    """A device-resident mesh: pattern, maps and element data (Sec. 3.2.2).

    cell: "tri" | "tet" | "quad" | "hex"; order 1..3; coords float64 [NV, d];
    cells int [NC, nv] in reference vertex order; elem_prec "fp64" | "fp32".
    """

    def __init__(self, cell, order, coords, cells, E0=1.0, Emin=1e-9, nu=0.3, p=3.0,
                 plane_strain=False, elem_prec="fp64", stream=None):
        L = N.lib()
        coords = np.ascontiguousarray(coords, np.float64)
        cells = np.ascontiguousarray(cells, np.int32)
        self.cell, self.order = cell, int(order)
        self.dim = coords.shape[1]
        self.material = N.Material(E0, Emin, nu, p, int(bool(plane_strain)))
        self.elem_prec = elem_prec
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        N.check(L.soptx_mesh_create(self.dim, N.CELL[cell], self.order, coords.shape[0],
                                    coords.ctypes.data_as(ctypes.c_void_p), cells.shape[0],
                                    cells.ctypes.data_as(ctypes.c_void_p) if cells.size else None,
                                    ctypes.byref(self.material), N.PREC[elem_prec], _stream(stream),
                                    ctypes.byref(h)))
        self._h = h
        ndof, nnz, nc, ldof = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        N.check(L.soptx_mesh_info(h, ctypes.byref(ndof), ctypes.byref(nnz), ctypes.byref(nc), ctypes.byref(ldof)))
        self.ndof, self.nnz, self.n_cells, self.ldof = ndof.value, nnz.value, nc.value, ldof.value
        self.nb = self.ldof // self.dim
        path, nbytes = ctypes.c_int32(), ctypes.c_int64()
        N.check(L.soptx_mesh_path(h, ctypes.byref(path)))
        N.check(L.soptx_mesh_device_bytes(h, ctypes.byref(nbytes)))
        self.path = N.PATH[path.value]
        self.device_bytes = nbytes.value
        ra, rs = ctypes.c_int32(), ctypes.c_int32()
        N.check(L.soptx_mesh_routes(h, ctypes.byref(ra), ctypes.byref(rs)))
        # the kernels serving the per-call work (soptx_mesh_routes)
        self.routes = {"assembly": ("lattice", "gather", "contract", "pairs")[ra.value],
                       "sensitivity": ("lattice", "gather", "strain")[rs.value]}

    @classmethod
    def from_workload(cls, wl, elem_prec=None, stream=None):
        return cls(wl.cell, wl.order, wl.coords, wl.cells, wl.E0, wl.Emin, wl.nu, wl.p, wl.plane_strain,
                   elem_prec or wl.elem_prec, stream)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib().soptx_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ structure
    def pattern(self, stream=None):
        indptr = torch.empty(self.ndof + 1, dtype=torch.int64, device=self.device)
        indices = torch.empty(self.nnz, dtype=torch.int32, device=self.device)
        N.check(N.lib().soptx_mesh_copy_pattern(self._h, ctypes.c_void_p(indptr.data_ptr()),
                                                ctypes.c_void_p(indices.data_ptr()), _stream(stream)))
        return indptr, indices

    def cell_nodes(self, stream=None):
        out = torch.empty((self.n_cells, self.nb), dtype=torch.int32, device=self.device)
        if self.n_cells:
            N.check(N.lib().soptx_mesh_copy_cell_nodes(self._h, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    # ------------------------------------------------------------ hot path
    def assemble_K(self, rho, vals=None, stream=None):
        if vals is None:
            vals = torch.empty(self.nnz, dtype=torch.float64, device=self.device)
        N.check(N.lib().soptx_assemble_K(self._h, _dptr(rho, torch.float64, self.n_cells, "rho"),
                                         _dptr(vals, torch.float64, self.nnz, "vals"), _stream(stream)))
        return vals

    def sensitivity(self, rho, u, dc=None, c=None, want_c=True, stream=None):
        if dc is None:
            dc = torch.empty(self.n_cells, dtype=torch.float64, device=self.device)
        if want_c and c is None:
            c = torch.empty(1, dtype=torch.float64, device=self.device)
        N.check(N.lib().soptx_sensitivity(self._h, _dptr(rho, torch.float64, self.n_cells, "rho"),
                                          _dptr(u, torch.float64, self.ndof, "u"),
                                          _dptr(dc, torch.float64, self.n_cells, "dc"),
                                          _dptr(c, torch.float64, 1, "c") if want_c else None, _stream(stream)))
        return dc, (c if want_c else None)

    def step(self, rho, u, vals=None, dc=None, c=None, stream=None):
        """K(rho), dc and c in one call (the per-iteration hot path)."""
        if vals is None:
            vals = torch.empty(self.nnz, dtype=torch.float64, device=self.device)
        if dc is None:
            dc = torch.empty(self.n_cells, dtype=torch.float64, device=self.device)
        if c is None:
            c = torch.empty(1, dtype=torch.float64, device=self.device)
        N.check(N.lib().soptx_assemble_and_sensitivity(
            self._h, _dptr(rho, torch.float64, self.n_cells, "rho"), _dptr(u, torch.float64, self.ndof, "u"),
            _dptr(vals, torch.float64, self.nnz, "vals"), _dptr(dc, torch.float64, self.n_cells, "dc"),
            _dptr(c, torch.float64, 1, "c"), _stream(stream)))
        return vals, dc, c

    def step_host(self, rho, u, vals=None, dcc=None, stream=None):
        """The step from host memory (soptx_step_host): rho [NC] and u [ndof]
        are CPU float64 tensors (pinned for asynchronous copies); returns
        (vals on the device, dc, c) with dc and c views of one host buffer
        dcc [NC + 1] (pinned when made here), valid once the stream has
        completed."""
        if vals is None:
            vals = torch.empty(self.nnz, dtype=torch.float64, device=self.device)
        if dcc is None:
            dcc = torch.empty(self.n_cells + 1, dtype=torch.float64, pin_memory=True)
        _hptr(dcc, self.n_cells + 1, "dcc")
        base = dcc.data_ptr()
        N.check(N.lib().soptx_step_host(
            self._h, _hptr(rho, self.n_cells, "rho"), _hptr(u, self.ndof, "u"),
            _dptr(vals, torch.float64, self.nnz, "vals"), ctypes.c_void_p(base),
            ctypes.c_void_p(base + 8 * self.n_cells), _stream(stream)))
        return vals, dcc[:self.n_cells], dcc[self.n_cells:]

    def compliance_vjp(self, rho, u, gout, want_u=True, stream=None):
        grad_rho = torch.empty(self.n_cells, dtype=torch.float64, device=self.device)
        grad_u = torch.empty(self.ndof, dtype=torch.float64, device=self.device) if want_u else None
        N.check(N.lib().soptx_compliance_vjp(
            self._h, _dptr(rho, torch.float64, self.n_cells, "rho"), _dptr(u, torch.float64, self.ndof, "u"),
            _dptr(gout, torch.float64, 1, "gout"), _dptr(grad_rho, torch.float64, self.n_cells, "grad_rho"),
            _dptr(grad_u, torch.float64, self.ndof, "grad_u") if want_u else None, _stream(stream)))
        return grad_rho, grad_u


    # ------------------------------------------------------------ the step after assembly
    def spmv(self, vals, x, y=None, stream=None):
        """y = K x with the CSR values `vals` (e.g. from assemble_K)."""
        if y is None:
            y = torch.empty(self.ndof, dtype=torch.float64, device=self.device)
        N.check(N.lib().soptx_spmv(self._h, _dptr(vals, torch.float64, self.nnz, "vals"),
                                   _dptr(x, torch.float64, self.ndof, "x"), _dptr(y, torch.float64, self.ndof, "y"),
                                   _stream(stream)))
        return y

    def solve(self, vals, fixed, f, u_fixed=None, rtol=1e-10, max_iter=10000, check_every=10, u0=None,
              stream=None):
        """K u = f on the free dofs (fixed: bool/uint8 [ndof]; u = u_fixed on the
        constrained ones, 0 if not given) by Jacobi-preconditioned CG from 0, or
        from the free entries of u0.  Returns (u, dict(iterations, converged,
        rel_residual))."""
        fixed = fixed.to(device=self.device, dtype=torch.uint8).contiguous()
        u = torch.zeros(self.ndof, dtype=torch.float64, device=self.device) if u_fixed is None else \
            u_fixed.to(device=self.device, dtype=torch.float64).clone().contiguous()
        if u0 is not None:
            u = torch.where(fixed.bool(), u, u0.to(device=self.device, dtype=torch.float64)).contiguous()
        opts = N.CgOpts(float(rtol), int(max_iter), int(check_every), int(u0 is not None))
        res = N.CgResult()
        N.check(N.lib().soptx_solve_cg(self._h, _dptr(vals, torch.float64, self.nnz, "vals"),
                                       _dptr(fixed, torch.uint8, self.ndof, "fixed"),
                                       _dptr(f, torch.float64, self.ndof, "f"),
                                       _dptr(u, torch.float64, self.ndof, "u"), ctypes.byref(opts), _stream(stream),
                                       ctypes.byref(res)))
        return u, dict(iterations=res.iterations, converged=bool(res.converged), rel_residual=res.rel_residual)


def step_group(meshes, rhos, us, stream=None):
    """The one-call step for several distinct meshes (soptx_assemble_and_sensitivity_group):
    small 2D and 3D box lattices share one kernel launch, the others get the
    ordinary call on the same stream.  Returns [(vals, dc, c)] in order, bitwise the
    results of each mesh's own step."""
    n = len(meshes)
    if not (len(rhos) == n and len(us) == n):
        raise ValueError("meshes, rhos and us must have the same length")
    outs = []
    P = ctypes.c_void_p * max(n, 1)
    hm, pr, pu, pv, pd, pc = P(), P(), P(), P(), P(), P()
    for k, (m, rho, u) in enumerate(zip(meshes, rhos, us)):
        vals = torch.empty(m.nnz, dtype=torch.float64, device=m.device)
        dc = torch.empty(m.n_cells, dtype=torch.float64, device=m.device)
        c = torch.empty(1, dtype=torch.float64, device=m.device)
        hm[k] = m._h.value
        pr[k] = _dptr(rho, torch.float64, m.n_cells, "rho").value
        pu[k] = _dptr(u, torch.float64, m.ndof, "u").value
        pv[k] = _dptr(vals, torch.float64, m.nnz, "vals").value
        pd[k] = _dptr(dc, torch.float64, m.n_cells, "dc").value
        pc[k] = _dptr(c, torch.float64, 1, "c").value
        outs.append((vals, dc, c))
    N.check(N.lib().soptx_assemble_and_sensitivity_group(n, hm, pr, pu, pv, pd, pc, _stream(stream)))
    return outs


def version():
    return N.lib().soptx_version().decode()


def host_plan(cell, order, coords, cells):
    """Host-only numbering and pattern (no GPU needed):
    returns dict(ndof, nnz, nb, path, indptr, indices, cell_nodes) as numpy arrays."""
    L = N.lib()
    coords = np.ascontiguousarray(coords, np.float64)
    cells = np.ascontiguousarray(cells, np.int32)
    dim = coords.shape[1]
    ndof, nnz, nb, path = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    args = [dim, N.CELL[cell], int(order), coords.shape[0], coords.ctypes.data_as(ctypes.c_void_p), cells.shape[0],
            cells.ctypes.data_as(ctypes.c_void_p) if cells.size else None]
    N.check(L.soptx_host_plan(*args, ctypes.byref(ndof), ctypes.byref(nnz), ctypes.byref(nb), ctypes.byref(path),
                              None, None, None))
    indptr = np.zeros(ndof.value + 1, np.int64)
    indices = np.zeros(max(nnz.value, 1), np.int32)
    cn = np.zeros((cells.shape[0], nb.value), np.int32)
    N.check(L.soptx_host_plan(*args, None, None, None, None, indptr.ctypes.data_as(ctypes.c_void_p),
                              indices.ctypes.data_as(ctypes.c_void_p), cn.ctypes.data_as(ctypes.c_void_p)))
    return dict(ndof=ndof.value, nnz=nnz.value, nb=nb.value, path=N.PATH[path.value], indptr=indptr,
                indices=indices[: nnz.value], cell_nodes=cn)


def host_pair_tables(cell, order, coords, cells, local_pair_bytes=False):
    """Host-only node-pair schedule of the pair kernel (no GPU needed): returns
    None for a mesh past the tables' limits, else dict(n_tiles, tile_offsets,
    pair_block, pair_block_t, pair_meta, record_cell, record_pair) as numpy arrays."""
    L = N.lib()
    coords = np.ascontiguousarray(coords, np.float64)
    cells = np.ascontiguousarray(cells, np.int32)
    args = [coords.shape[1], N.CELL[cell], int(order), coords.shape[0], coords.ctypes.data_as(ctypes.c_void_p),
            cells.shape[0], cells.ctypes.data_as(ctypes.c_void_p) if cells.size else None, int(bool(local_pair_bytes))]
    nt, nr = ctypes.c_int64(), ctypes.c_int64()
    N.check(L.soptx_host_pair_tables(*args, ctypes.byref(nt), ctypes.byref(nr), None, None, None, None, None, None))
    if nt.value < 0:
        return None
    lanes = max(nt.value, 1) * 32
    out = dict(n_tiles=nt.value, tile_offsets=np.zeros(nt.value + 1, np.uint32),
               pair_block=np.zeros(lanes, np.uint32), pair_block_t=np.zeros(lanes, np.uint32),
               pair_meta=np.zeros(lanes, np.uint32), record_cell=np.zeros(max(nr.value, 1), np.int32),
               record_pair=np.zeros(max(nr.value, 1), np.uint16))
    ptr = lambda k: out[k].ctypes.data_as(ctypes.c_void_p)
    N.check(L.soptx_host_pair_tables(*args, None, None, ptr("tile_offsets"), ptr("pair_block"), ptr("pair_block_t"),
                                     ptr("pair_meta"), ptr("record_cell"), ptr("record_pair")))
    for k in ("pair_block", "pair_block_t", "pair_meta"):
        out[k] = out[k][: nt.value * 32]
    for k in ("record_cell", "record_pair"):
        out[k] = out[k][: nr.value]
    return out


def host_row_tables(cell, order, coords, cells):
    """Host-only node-owner schedule of 3D meshes with FP32 element matrices (no
    GPU needed): None where mesh creation builds none, else dict(nb, node_records
    int32 [nn][4], chain_cell, chain_local, lane_records [n_incidences][nb])."""
    L = N.lib()
    coords = np.ascontiguousarray(coords, np.float64)
    cells = np.ascontiguousarray(cells, np.int32)
    args = [coords.shape[1], N.CELL[cell], int(order), coords.shape[0], coords.ctypes.data_as(ctypes.c_void_p),
            cells.shape[0], cells.ctypes.data_as(ctypes.c_void_p) if cells.size else None]
    nn, ni, nb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    N.check(L.soptx_host_row_tables(*args, ctypes.byref(nn), ctypes.byref(ni), ctypes.byref(nb), None, None, None,
                                    None))
    if nn.value < 0:
        return None
    out = dict(nb=nb.value, node_records=np.zeros((max(nn.value, 1), 4), np.int32),
               chain_cell=np.zeros(max(ni.value, 1), np.int32), chain_local=np.zeros(max(ni.value, 1), np.uint8),
               lane_records=np.zeros((max(ni.value, 1), nb.value), np.uint16))
    ptr = lambda k: out[k].ctypes.data_as(ctypes.c_void_p)
    N.check(L.soptx_host_row_tables(*args, None, None, None, ptr("node_records"), ptr("chain_cell"),
                                    ptr("chain_local"), ptr("lane_records")))
    out["node_records"] = out["node_records"][: nn.value]
    for k in ("chain_cell", "chain_local", "lane_records"):
        out[k] = out[k][: ni.value]
    return out
