"""ctypes declarations of the C ABI in include/soptx.h (argument marshalling only).

The library is the in-tree ``libsoptx.so`` built by ``build.py``.  There is no
fallback: if the library is missing or fails to load, every call raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsoptx.so")

STATUS = {0: "SOPTX_OK", 1: "SOPTX_EINVAL", 2: "SOPTX_ENOMEM", 3: "SOPTX_ECUDA", 4: "SOPTX_EBUSY",
          5: "SOPTX_ETIMEOUT", 6: "SOPTX_ENOTFOUND", 7: "SOPTX_EINTERNAL"}
CELL = {"tri": 0, "tet": 1, "quad": 2, "hex": 3}
PREC = {"fp64": 0, "fp32": 1}
PATH = {0: "lattice", 1: "uniform", 2: "cached"}

# Every exported symbol of include/soptx.h: name -> (restype, argtypes)
P, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
PP = ctypes.POINTER(ctypes.c_void_p)
Pi64 = ctypes.POINTER(ctypes.c_int64)
Pi32 = ctypes.POINTER(ctypes.c_int32)


class Material(ctypes.Structure):
    _fields_ = [("E0", ctypes.c_double), ("Emin", ctypes.c_double), ("nu", ctypes.c_double),
                ("p", ctypes.c_double), ("plane_strain", ctypes.c_int32)]


class CgOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("warm_start", ctypes.c_int32)]


class CgResult(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32), ("rel_residual", ctypes.c_double)]


class OcOpts(ctypes.Structure):
    _fields_ = [("volfrac", ctypes.c_double), ("move", ctypes.c_double), ("eta", ctypes.c_double),
                ("l_lo", ctypes.c_double), ("l_hi", ctypes.c_double), ("tol", ctypes.c_double)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_cap_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int32), ("n_streams", ctypes.c_int32),
                ("max_queue", ctypes.c_int32), ("device", ctypes.c_int32), ("group_small", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("job", ctypes.c_uint64), ("dim", ctypes.c_int32), ("cell", ctypes.c_int32),
                ("order", ctypes.c_int32), ("n_vertices", ctypes.c_int64), ("coords", ctypes.c_void_p),
                ("n_cells", ctypes.c_int64), ("cell_vertices", ctypes.c_void_p), ("mat", Material),
                ("prec", ctypes.c_int32), ("d_rho", ctypes.c_void_p), ("d_u", ctypes.c_void_p),
                ("d_vals", ctypes.c_void_p), ("d_dc", ctypes.c_void_p), ("d_c", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("queue_us", ctypes.c_double), ("latency_us", ctypes.c_double),
                ("gpu_us", ctypes.c_double), ("nnz", ctypes.c_int64), ("mesh_was_resident", ctypes.c_int32),
                ("gpu_start_us", ctypes.c_double), ("gpu_end_us", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("evictions", ctypes.c_int64), ("mesh_setups", ctypes.c_int64), ("resident_bytes", ctypes.c_int64),
                ("peak_resident_bytes", ctypes.c_int64), ("resident_meshes", ctypes.c_int32),
                ("in_flight", ctypes.c_int32), ("queued", ctypes.c_int32), ("groups", ctypes.c_int64)]


class PipeRates(ctypes.Structure):
    _fields_ = [("ffma_per_s", ctypes.c_double), ("dfma_per_s", ctypes.c_double), ("f2f64_per_s", ctypes.c_double),
                ("sms", ctypes.c_int32)]


SIGNATURES = {
    "soptx_mesh_create": (i32, [i32, i32, i32, i64, P, i64, P, ctypes.POINTER(Material), i32, P, PP]),
    "soptx_mesh_info": (i32, [P, Pi64, Pi64, Pi64, Pi32]),
    "soptx_mesh_pattern": (i32, [P, PP, PP]),
    "soptx_mesh_cell_nodes": (i32, [P, PP, Pi32]),
    "soptx_mesh_copy_pattern": (i32, [P, P, P, P]),
    "soptx_mesh_copy_cell_nodes": (i32, [P, P, P]),
    "soptx_mesh_path": (i32, [P, Pi32]),
    "soptx_mesh_device_bytes": (i32, [P, Pi64]),
    "soptx_mesh_routes": (i32, [P, Pi32, Pi32]),
    "soptx_assemble_K": (i32, [P, P, P, P]),
    "soptx_sensitivity": (i32, [P, P, P, P, P, P]),
    "soptx_assemble_and_sensitivity": (i32, [P, P, P, P, P, P, P]),
    "soptx_assemble_and_sensitivity_group": (i32, [i32, P, P, P, P, P, P, P]),
    "soptx_step_host": (i32, [P, P, P, P, P, P, P]),
    "soptx_compliance_vjp": (i32, [P, P, P, P, P, P, P]),
    "soptx_mesh_destroy": (i32, [P]),
    "soptx_host_plan": (i32, [i32, i32, i32, i64, P, i64, P, Pi64, Pi64, Pi32, Pi32, P, P, P]),
    "soptx_host_pair_tables": (i32, [i32, i32, i32, i64, P, i64, P, i32, Pi64, Pi64, P, P, P, P, P, P]),
    "soptx_host_row_tables": (i32, [i32, i32, i32, i64, P, i64, P, Pi64, Pi64, Pi32, P, P, P, P]),
    "soptx_lattice_sensitivity_noalloc": (i32, [i32, P, P, ctypes.POINTER(Material), P, P, P, P, P]),
    "soptx_spmv": (i32, [P, P, P, P, P]),
    "soptx_solve_cg": (i32, [P, P, P, P, P, ctypes.POINTER(CgOpts), P, ctypes.POINTER(CgResult)]),
    "soptx_filter_create": (i32, [i32, i64, P, P, ctypes.c_double, P, PP]),
    "soptx_filter_info": (i32, [P, Pi64, Pi64]),
    "soptx_filter_sensitivity": (i32, [P, P, P, P, P]),
    "soptx_filter_density": (i32, [P, P, P, P]),
    "soptx_filter_density_grad": (i32, [P, P, P, P]),
    "soptx_filter_destroy": (i32, [P]),
    "soptx_heaviside": (i32, [i64, ctypes.c_double, P, P, P, P]),
    "soptx_oc_update": (i32, [i64, P, P, P, P, ctypes.POINTER(OcOpts), P, P, P]),
    "soptx_server_create": (i32, [ctypes.POINTER(ServerOpts), PP]),
    "soptx_serve_submit": (i32, [P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "soptx_serve_mesh_bytes_bound": (i32, [ctypes.POINTER(Request), Pi64]),
    "soptx_serve_wait": (i32, [P, ctypes.c_uint64, i64, ctypes.POINTER(Result)]),
    "soptx_serve_poll": (i32, [P, ctypes.c_uint64, Pi32]),
    "soptx_server_stats_get": (i32, [P, ctypes.POINTER(ServerStats)]),
    "soptx_server_destroy": (i32, [P]),
    "soptx_last_error": (ctypes.c_char_p, []),
    "soptx_version": (ctypes.c_char_p, []),
    "soptx_measure_pipe_rates": (i32, [ctypes.POINTER(PipeRates)]),
    "soptx_debug_fail_alloc_after": (None, [i64]),
    "soptx_debug_lattice_no_sectors": (None, [i32]),
}

_lib = None


class SoptxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, str(code)), msg))
        self.code = code


def lib():
    """Load libsoptx.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsoptx.so is not built (run paper_2505_02438_gb300.build.build_library())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code):
    if code != 0:
        raise SoptxError(code, lib().soptx_last_error().decode(errors="replace"))
