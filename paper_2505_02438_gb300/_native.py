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


SIGNATURES = {
    "soptx_mesh_create": (i32, [i32, i32, i32, i64, P, i64, P, ctypes.POINTER(Material), i32, P, PP]),
    "soptx_mesh_info": (i32, [P, Pi64, Pi64, Pi64, Pi32]),
    "soptx_mesh_pattern": (i32, [P, PP, PP]),
    "soptx_mesh_cell_nodes": (i32, [P, PP, Pi32]),
    "soptx_mesh_copy_pattern": (i32, [P, P, P, P]),
    "soptx_mesh_copy_cell_nodes": (i32, [P, P, P]),
    "soptx_mesh_path": (i32, [P, Pi32]),
    "soptx_mesh_device_bytes": (i32, [P, Pi64]),
    "soptx_assemble_K": (i32, [P, P, P, P]),
    "soptx_sensitivity": (i32, [P, P, P, P, P, P]),
    "soptx_assemble_and_sensitivity": (i32, [P, P, P, P, P, P, P]),
    "soptx_compliance_vjp": (i32, [P, P, P, P, P, P, P]),
    "soptx_mesh_destroy": (i32, [P]),
    "soptx_host_plan": (i32, [i32, i32, i32, i64, P, i64, P, Pi64, Pi64, Pi32, Pi32, P, P, P]),
    "soptx_lattice_sensitivity_noalloc": (i32, [i32, P, P, ctypes.POINTER(Material), P, P, P, P, P]),
    "soptx_last_error": (ctypes.c_char_p, []),
    "soptx_version": (ctypes.c_char_p, []),
    "soptx_debug_fail_alloc_after": (None, [i64]),
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
