"""Python handle on the continuous-batching server of include/soptx_serve.h.

The server keeps each design job's mesh resident, admits requests in arrival
order as slots and HBM budget allow, and overlaps their kernels on a stream
pool; this module only marshals requests and results."""
import ctypes

import numpy as np
import torch

from . import _native as N
from .api import _dptr


def _cuda_f64(t, name):
    """A contiguous FP64 CUDA tensor whose length only the mesh fixes (u holds
    ndof values, vals nnz: the caller sizes them from the job's mesh)."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("%s must be a contiguous torch.float64 tensor" % name)
    return ctypes.c_void_p(t.data_ptr())


def _mesh_request(wl, coords, cells):
    """A request whose mesh description is the workload's (device buffers unset)."""
    r = N.Request()
    r.dim = coords.shape[1]
    r.cell = N.CELL[wl.cell]
    r.order = int(wl.order)
    r.n_vertices = coords.shape[0]
    r.coords = coords.ctypes.data_as(ctypes.c_void_p)
    r.n_cells = cells.shape[0]
    r.cell_vertices = cells.ctypes.data_as(ctypes.c_void_p)
    r.mat = N.Material(wl.E0, wl.Emin, wl.nu, wl.p, int(wl.plane_strain))
    r.prec = N.PREC[getattr(wl, "elem_prec", "fp64")]
    return r


def mesh_bytes_bound(wl):
    """The device bytes the server makes room for before it builds the mesh of
    the workload `wl` (an upper bound of soptx_mesh_create's; host only)."""
    coords = np.ascontiguousarray(wl.coords, np.float64)
    cells = np.ascontiguousarray(wl.cells, np.int32)
    b = ctypes.c_int64()
    N.check(N.lib().soptx_serve_mesh_bytes_bound(ctypes.byref(_mesh_request(wl, coords, cells)), ctypes.byref(b)))
    return b.value


class Server:
    def __init__(self, hbm_cap_bytes=120 << 30, max_slots=16, n_streams=8, max_queue=4096, device=None,
                 group_small=True):
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = torch.device("cuda", dev)
        opts = N.ServerOpts(int(hbm_cap_bytes), int(max_slots), int(n_streams), int(max_queue), dev,
                            1 if group_small else 0)
        h = ctypes.c_void_p()
        N.check(N.lib().soptx_server_create(ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, job, wl, rho, u, vals=None, dc=None, c=None):
        """Queue one iteration of design `job` (mesh and material from the
        workload `wl`); returns a ticket.  Outputs are allocated if not given."""
        coords = np.ascontiguousarray(wl.coords, np.float64)
        cells = np.ascontiguousarray(wl.cells, np.int32)
        nc = cells.shape[0]
        if dc is None:
            dc = torch.empty(nc, dtype=torch.float64, device=self.device)
        if c is None:
            c = torch.empty(1, dtype=torch.float64, device=self.device)
        r = _mesh_request(wl, coords, cells)
        r.job = int(job)
        r.d_rho = _dptr(rho, torch.float64, nc, "rho")
        r.d_u = _cuda_f64(u, "u")
        r.d_vals = _cuda_f64(vals, "vals") if vals is not None else None
        r.d_dc = _dptr(dc, torch.float64, nc, "dc")
        r.d_c = _dptr(c, torch.float64, 1, "c")
        t = ctypes.c_uint64()
        N.check(N.lib().soptx_serve_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        self._keep[t.value] = (coords, cells, rho, u, vals, dc, c)
        return t.value

    def outputs(self, ticket):
        coords, cells, rho, u, vals, dc, c = self._keep[ticket]
        return vals, dc, c

    def wait(self, ticket, timeout_us=-1):
        res = N.Result()
        N.check(N.lib().soptx_serve_wait(self._h, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(res)))
        out = dict(status=res.status, queue_us=res.queue_us, latency_us=res.latency_us, gpu_us=res.gpu_us,
                   nnz=res.nnz, mesh_was_resident=bool(res.mesh_was_resident), gpu_start_us=res.gpu_start_us,
                   gpu_end_us=res.gpu_end_us)
        vals, dc, c = self.outputs(ticket)
        out.update(vals=vals, dc=dc, c=c)
        del self._keep[ticket]
        return out

    def poll(self, ticket):
        d = ctypes.c_int32()
        N.check(N.lib().soptx_serve_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(d)))
        return bool(d.value)

    def stats(self):
        st = N.ServerStats()
        N.check(N.lib().soptx_server_stats_get(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in N.ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib().soptx_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def overlap(results):
    """How much the requests' device intervals [gpu_start_us, gpu_end_us]
    overlapped: the largest number in flight at one instant, and the share of
    requests whose interval intersects another's."""
    iv = sorted((r["gpu_start_us"], r["gpu_end_us"]) for r in results if r["gpu_end_us"] > r["gpu_start_us"])
    ev = sorted([(a, 1) for a, _ in iv] + [(b, -1) for _, b in iv], key=lambda t: (t[0], t[1]))
    cur = peak = 0
    for _, d in ev:
        cur += d
        peak = max(peak, cur)
    shared = 0
    end_max = -np.inf
    for k, (a, b) in enumerate(iv):
        # intersects an earlier interval, or the next one starts before this ends
        if a < end_max or (k + 1 < len(iv) and iv[k + 1][0] < b):
            shared += 1
        end_max = max(end_max, b)
    return {"max_in_flight": peak, "overlapped_share": shared / max(1, len(iv))}

