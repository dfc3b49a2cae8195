"""ctypes mirror of include/ib.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

IB_OK, IB_EINVAL, IB_ENOMEM, IB_ESTATE, IB_ENOCONV, IB_EBREAKDOWN, IB_ECUDA, IB_ETIMEOUT = range(8)
STATUS_NAMES = {0: "IB_OK", 1: "IB_EINVAL", 2: "IB_ENOMEM", 3: "IB_ESTATE", 4: "IB_ENOCONV",
                5: "IB_EBREAKDOWN", 6: "IB_ECUDA", 7: "IB_ETIMEOUT"}
IB_INLET_VELOCITY, IB_OUTLET_ZERO_P, IB_INLET_PRESSURE = 0, 1, 2
IB_VISCOUS_GRAD, IB_VISCOUS_SYM = 0, 1
IB_FP64, IB_MIXED = 0, 1
IB_PC_MULTIGRID, IB_PC_JACOBI = 0, 1
IB_MAX_PORTS, IB_MAX_HARMONICS, IB_MAX_LEVEL = 8, 8, 3
IB_TUNE_N = 5
IB_TANGENTIAL_FREE, IB_TANGENTIAL_ZERO = 0, 1
TUNE_INDEX = {"poisson_kernel": 0, "stream_chunk": 1, "mg_small": 2, "mg_sweeps": 3, "mg_persist": 4}

FIELD = {
    "U": 0, "P": 1, "PHI": 2, "U_TENT": 3, "U_IB": 4, "F_LAG": 5, "B_F": 6, "NODE_Q": 7,
    "NODE_FLAGS": 8, "ACTIVE": 9, "LEVEL": 10, "IB_ORIGIN": 11, "IB_WEIGHTS": 12, "IB_FREE": 13,
}

EXPORTS = ("ib_grid_create", "ib_set_boundary", "ipcs_step", "ib_fields_get", "ib_fields_set",
           "ib_grid_info", "ib_last_error", "ib_grid_destroy", "ib_batch_create", "ib_batch_step",
           "ib_batch_fields_get", "ib_batch_info", "ib_batch_last_error", "ib_batch_destroy",
           "ib_fields_get_noalloc", "ib_set_points", "ib_wss")

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class IbPort(C.Structure):
    _fields_ = [
        ("axis", C.c_int32), ("side", C.c_int32), ("center", C.c_double * 3), ("radius", C.c_double),
        ("kind", C.c_int32), ("profile", C.c_int32), ("n_harm", C.c_int32),
        ("a0", C.c_double), ("a", C.c_double * IB_MAX_HARMONICS), ("b", C.c_double * IB_MAX_HARMONICS),
        ("period", C.c_double),
    ]


class IbGridDesc(C.Structure):
    _fields_ = [
        ("origin", C.c_double * 3), ("extent", C.c_double * 3), ("n", C.c_int32 * 3),
        ("max_level", C.c_int32), ("refine_band", C.c_int32), ("reduce_band", C.c_int32),
        ("nu", C.c_double), ("rho", C.c_double), ("dt", C.c_double), ("precision", C.c_int32),
        ("rtol_mom", C.c_double), ("rtol_p", C.c_double), ("rtol_corr", C.c_double), ("rtol_ib", C.c_double),
        ("max_iter", C.c_int32), ("profile", C.c_int32), ("deferred", C.c_int32), ("poisson_pc", C.c_int32),
        ("viscous_form", C.c_int32),
        ("n_ports", C.c_int32), ("ports", IbPort * IB_MAX_PORTS),
        ("stream", C.c_void_p), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_ctx", C.c_void_p),
        ("tune", C.c_int32 * IB_TUNE_N), ("port_tangential", C.c_int32),
    ]


class IbInfo(C.Structure):
    _fields_ = [
        ("n_nodes", C.c_int64), ("n_dof", C.c_int64), ("n_hanging", C.c_int64), ("n_leaf_cells", C.c_int64),
        ("n_leaf_cells_level", C.c_int64 * (IB_MAX_LEVEL + 1)), ("n_active_coarse", C.c_int64),
        ("n_bricks", C.c_int64), ("n_slots", C.c_int64), ("n_interface", C.c_int64), ("n_points", C.c_int64),
        ("af_nnz", C.c_int64), ("a_ratio", C.c_double * 3), ("step", C.c_int64), ("time", C.c_double),
        ("iters_mom", C.c_int32 * 3), ("iters_ib", C.c_int32), ("iters_p", C.c_int32),
        ("iters_corr", C.c_int32 * 3), ("outer_mom", C.c_int32), ("outer_p", C.c_int32),
        ("outer_corr", C.c_int32), ("res_mom", C.c_double), ("res_ib", C.c_double), ("res_p", C.c_double),
        ("res_corr", C.c_double), ("status_mom", C.c_int32), ("status_ib", C.c_int32), ("status_p", C.c_int32),
        ("status_corr", C.c_int32), ("device_bytes", C.c_int64), ("n_valid_slots", C.c_int64),
        ("prof_ms", C.c_double * 12), ("prof_launches", C.c_int64 * 12), ("kernel_launches", C.c_int64),
        ("mg_levels", C.c_int32), ("mg_coarsest", C.c_int32),
    ]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out


def bind(lib: C.CDLL) -> C.CDLL:
    """Declare argument and return types of every exported entry point."""
    P = C.POINTER
    lib.ib_grid_create.argtypes = [P(IbGridDesc), P(C.c_void_p)]
    lib.ib_grid_create.restype = C.c_int
    lib.ib_set_boundary.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.ib_set_boundary.restype = C.c_int
    lib.ipcs_step.argtypes = [C.c_void_p, C.c_int32]
    lib.ipcs_step.restype = C.c_int
    lib.ib_fields_get.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t, C.c_int32]
    lib.ib_fields_get.restype = C.c_int
    lib.ib_fields_get_noalloc.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t, C.c_int32]
    lib.ib_fields_get_noalloc.restype = C.c_int
    lib.ib_fields_set.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t, C.c_int32]
    lib.ib_fields_set.restype = C.c_int
    lib.ib_set_points.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int32]
    lib.ib_set_points.restype = C.c_int
    lib.ib_wss.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
    lib.ib_wss.restype = C.c_int
    lib.ib_grid_info.argtypes = [C.c_void_p, P(IbInfo)]
    lib.ib_grid_info.restype = C.c_int
    lib.ib_last_error.argtypes = [C.c_void_p]
    lib.ib_last_error.restype = C.c_char_p
    lib.ib_grid_destroy.argtypes = [C.c_void_p]
    lib.ib_grid_destroy.restype = None
    lib.ib_batch_create.argtypes = [P(C.c_void_p), C.c_int32, P(C.c_void_p)]
    lib.ib_batch_create.restype = C.c_int
    lib.ib_batch_step.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
    lib.ib_batch_step.restype = C.c_int
    lib.ib_batch_fields_get.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_size_t, C.c_int32]
    lib.ib_batch_fields_get.restype = C.c_int
    lib.ib_batch_info.argtypes = [C.c_void_p, C.c_int32, P(IbInfo)]
    lib.ib_batch_info.restype = C.c_int
    lib.ib_batch_last_error.argtypes = [C.c_void_p]
    lib.ib_batch_last_error.restype = C.c_char_p
    lib.ib_batch_destroy.argtypes = [C.c_void_p]
    lib.ib_batch_destroy.restype = None
    return lib


def library_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libibgpu.so")
