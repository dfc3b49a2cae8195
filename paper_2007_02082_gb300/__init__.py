"""GB300 IB-FE-IPCS: Python binding of the native library (include/ib.h).

Every step of the time integration runs in the library's CUDA kernels; this
module only marshals arguments.  There is no CPU fallback: if the library is
missing or no CUDA device is present, constructing a grid raises.

    from paper_2007_02082_gb300 import IBGrid
    g = IBGrid(case, precision="mixed")      # ib_grid_create + ib_set_boundary
    g.ipcs_step(10)                          # ipcs_step
    u = g.ib_fields_get("U")                 # ib_fields_get -> numpy
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _abi
from ._abi import FIELD, IB_FP64, IB_MIXED, STATUS_NAMES

_LIB = None


class IBError(RuntimeError):
    def __init__(self, call, status, msg):
        super().__init__(f"{call} -> {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load_library(build_if_missing: bool = False) -> C.CDLL:
    """Load lib/libibgpu.so (optionally building it first)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _abi.library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"native library not built: {path} (run __graft_entry__.build())")
        from .build import build
        build()
    _LIB = _abi.bind(C.CDLL(path))
    return _LIB


def _port_tangential(case):
    t = case.get("port_tangential", "free")
    if t not in ("free", "zero"):
        raise ValueError(f"port_tangential must be 'free' or 'zero', not {t!r}")
    return _abi.IB_TANGENTIAL_ZERO if t == "zero" else _abi.IB_TANGENTIAL_FREE


def _viscous_form(case):
    form = case.get("viscous", "grad")
    if form not in ("grad", "sym"):
        raise ValueError(f"viscous must be 'grad' or 'sym', not {form!r}")
    return _abi.IB_VISCOUS_SYM if form == "sym" else _abi.IB_VISCOUS_GRAD


def _port_struct(port):
    p = _abi.IbPort()
    p.axis, p.side = port["axis"], port["side"]
    for a in range(3):
        p.center[a] = port["center"][a]
    p.radius = port["radius"]
    kinds = {"inlet": _abi.IB_INLET_VELOCITY, "pinlet": _abi.IB_INLET_PRESSURE, "outlet": _abi.IB_OUTLET_ZERO_P}
    if port["kind"] not in kinds:
        raise ValueError(f"unknown port kind {port['kind']!r}")
    p.kind = kinds[port["kind"]]
    p.profile = 0
    p.a0 = port.get("a0", 0.0)
    a = list(port.get("a", ()))
    b = list(port.get("b", ()))
    p.n_harm = max(len(a), len(b))
    for k, v in enumerate(a):
        p.a[k] = v
    for k, v in enumerate(b):
        p.b[k] = v
    p.period = port.get("period", 1.0)
    return p


class _TorchAllocator:
    """Routes library allocations through PyTorch's caching allocator."""

    def __init__(self, device, stream):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream
        self.alloc = _abi.ALLOC_FN(self._alloc)
        self.free = _abi.FREE_FN(self._free)
        self.calls = 0          # device allocations the library asked for

    def _alloc(self, nbytes, ctx):
        self.calls += 1
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:
            return None

    def _free(self, ptr, ctx):
        try:
            self.torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass


class IBGrid:
    """One resident IB-FE-IPCS problem (an ib_grid handle)."""

    def __init__(self, case, precision="fp64", stream=None, torch_alloc=True, rtol=None, max_iter=0,
                 device=0, profile=False, deferred=False, poisson_pc="multigrid", tune=None):
        """tune: launch choices (ib_grid_desc.tune), a dict with any of
        "poisson_kernel" (1 staged, 2 register-pipelined, 3 persistent), "stream_chunk"
        (4 or 8), "mg_small" (nodes), "mg_sweeps" (1-4) and "mg_persist" (1
        separate launches, 2 one cooperative launch); None or 0 keeps
        the library's defaults (see paper_2007_02082_gb300.tune)."""
        self.lib = load_library()
        self.case = case
        self._alloc = None
        st = 0
        try:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("no CUDA device: the library has no CPU path")
            torch.cuda.set_device(device)
            s = stream if stream is not None else torch.cuda.current_stream(device)
            st = s.cuda_stream
            if torch_alloc:
                self._alloc = _TorchAllocator(device, s)
        except ImportError:
            if stream is not None:
                st = int(stream)
        d = _abi.IbGridDesc()
        for a in range(3):
            d.origin[a] = case["origin"][a]
            d.extent[a] = case["extent"][a]
            d.n[a] = case["n"][a]
        d.max_level = case["max_level"]
        d.refine_band = case["refine_band"]
        d.reduce_band = case["reduce_band"]
        d.nu, d.rho, d.dt = case["nu"], case["rho"], case["dt"]
        d.precision = IB_MIXED if precision == "mixed" else IB_FP64
        rt = rtol or {}
        d.rtol_mom = rt.get("mom", 0.0)
        d.rtol_p = rt.get("p", 0.0)
        d.rtol_corr = rt.get("corr", 0.0)
        d.rtol_ib = rt.get("ib", 0.0)
        d.max_iter = max_iter
        d.profile = 1 if profile else 0
        d.deferred = 1 if deferred else 0
        if poisson_pc not in ("multigrid", "jacobi"):
            raise ValueError("poisson_pc must be 'multigrid' or 'jacobi'")
        d.poisson_pc = _abi.IB_PC_JACOBI if poisson_pc == "jacobi" else _abi.IB_PC_MULTIGRID
        d.viscous_form = _viscous_form(case)
        d.port_tangential = _port_tangential(case)
        for k, v in (tune or {}).items():
            if k not in _abi.TUNE_INDEX:
                raise ValueError(f"unknown launch choice {k!r}")
            d.tune[_abi.TUNE_INDEX[k]] = int(v or 0)
        self.tune = dict(tune or {})
        d.n_ports = len(case["ports"])
        for k, port in enumerate(case["ports"]):
            d.ports[k] = _port_struct(port)
        d.stream = st
        if self._alloc is not None:
            d.dev_alloc = self._alloc.alloc
            d.dev_free = self._alloc.free
        self._desc = d
        h = C.c_void_p()
        s = self.lib.ib_grid_create(C.byref(d), C.byref(h))
        if s != 0:
            raise IBError("ib_grid_create", s, "invalid description")
        self.h = h
        X = np.ascontiguousarray(case["X"], dtype=np.float64)
        dS = np.ascontiguousarray(case["dS"], dtype=np.float64)
        UB = np.ascontiguousarray(case["UB"], dtype=np.float64)
        inside = np.ascontiguousarray(case["inside"], dtype=np.uint8)
        self.ib_set_boundary(X, dS, UB, inside)

    # -- C-ABI calls ---------------------------------------------------------
    def _check(self, call, s):
        if s != 0:
            raise IBError(call, s, self.lib.ib_last_error(self.h).decode())

    def ib_set_boundary(self, X, dS, UB, inside):
        self._keep = (X, dS, UB, inside)
        s = self.lib.ib_set_boundary(self.h, int(X.shape[0]), X.ctypes.data, dS.ctypes.data,
                                     UB.ctypes.data if UB is not None else None,
                                     inside.ctypes.data if inside is not None else None)
        self._check("ib_set_boundary", s)

    def ipcs_step(self, nsteps=1):
        self._check("ipcs_step", self.lib.ipcs_step(self.h, int(nsteps)))

    def ib_grid_info(self):
        info = _abi.IbInfo()
        self._check("ib_grid_info", self.lib.ib_grid_info(self.h, C.byref(info)))
        return info.as_dict()

    def _shape(self, field):
        info = self.ib_grid_info()
        N, M = info["n_nodes"], info["n_points"]
        n = self.case["n"]
        return {
            "U": ((N, 3), np.float64), "U_TENT": ((N, 3), np.float64), "U_IB": ((N, 3), np.float64),
            "P": ((N,), np.float64), "PHI": ((N,), np.float64), "F_LAG": ((M, 3), np.float64),
            "B_F": ((M, 3), np.float64), "NODE_Q": ((N, 3), np.int32), "NODE_FLAGS": ((N,), np.uint8),
            "ACTIVE": ((n[2], n[1], n[0]), np.uint8), "LEVEL": ((n[2], n[1], n[0]), np.uint8),
            "IB_ORIGIN": ((M, 3), np.int32), "IB_WEIGHTS": ((M, 64), np.float64), "IB_FREE": ((M, 64), np.uint8),
        }[field]

    def ib_fields_get(self, field, out=None):
        """Copy a field to a new host numpy array, or into `out`: a device
        tensor, or a host numpy array of the field's shape and dtype (for
        example pinned memory), which the library writes directly."""
        shape, dt = self._shape(field)
        if isinstance(out, np.ndarray):                  # host destination
            if out.shape != tuple(shape) or out.dtype != np.dtype(dt) or not out.flags.c_contiguous \
                    or not out.flags.writeable:
                raise ValueError(f"out must be a writable C-contiguous {np.dtype(dt)} array of shape {shape}")
            self._check("ib_fields_get", self.lib.ib_fields_get(self.h, FIELD[field], out.ctypes.data, out.nbytes, 0))
            return out
        if out is not None:                              # device tensor destination
            nbytes = out.numel() * out.element_size()
            self._check("ib_fields_get", self.lib.ib_fields_get(self.h, FIELD[field], C.c_void_p(out.data_ptr()),
                                                                nbytes, 1))
            return out
        arr = np.empty(shape, dtype=dt)
        self._check("ib_fields_get", self.lib.ib_fields_get(self.h, FIELD[field], arr.ctypes.data, arr.nbytes, 0))
        return arr

    def ib_fields_get_noalloc(self, field, out=None):
        """ib_fields_get_noalloc: U, P or PHI of a parked deferred handle, read
        through the library's fixed device scratch (no device allocation).
        `out`, if given, is a contiguous float64 CUDA tensor of the field's
        shape on the handle's device."""
        shape, dt = self._shape(field)
        if out is not None:
            import torch
            if (not out.is_cuda or out.dtype != torch.float64 or not out.is_contiguous()
                    or tuple(out.shape) != tuple(shape)):
                raise ValueError(f"out must be a contiguous float64 CUDA tensor of shape {shape}")
            nbytes = out.numel() * out.element_size()
            self._check("ib_fields_get_noalloc", self.lib.ib_fields_get_noalloc(
                self.h, FIELD[field], C.c_void_p(out.data_ptr()), nbytes, 1))
            return out
        arr = np.empty(shape, dtype=dt)
        self._check("ib_fields_get_noalloc",
                    self.lib.ib_fields_get_noalloc(self.h, FIELD[field], arr.ctypes.data, arr.nbytes, 0))
        return arr

    def ib_fields_set(self, field, values):
        shape, dt = self._shape(field)
        arr = np.ascontiguousarray(values, dtype=dt).reshape(shape)
        self._check("ib_fields_set", self.lib.ib_fields_set(self.h, FIELD[field], arr.ctypes.data, arr.nbytes, 0))

    def ib_set_points(self, X, UB=None):
        """Move the Lagrangian points (moving or deforming wall): X and U_B of
        shape (M, 3), numpy arrays or CUDA tensors; U_B None means a wall at
        rest.  The supports, weights, A_F and spreading lists are rebuilt on
        the device for the following steps."""
        if hasattr(X, "is_cuda") and X.is_cuda:
            import torch
            x = X.detach().to(torch.float64).contiguous().reshape(-1, 3)
            u = None if UB is None else UB.detach().to(device=x.device, dtype=torch.float64).contiguous().reshape(-1, 3)
            if u is not None and u.shape != x.shape:
                raise ValueError("X and UB differ in shape")
            self._check("ib_set_points", self.lib.ib_set_points(self.h, x.shape[0], C.c_void_p(x.data_ptr()),
                                                                None if u is None else C.c_void_p(u.data_ptr()), 1))
            return
        x = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
        u = None if UB is None else np.ascontiguousarray(UB, dtype=np.float64).reshape(-1, 3)
        if u is not None and u.shape != x.shape:
            raise ValueError("X and UB differ in shape")
        self._check("ib_set_points", self.lib.ib_set_points(self.h, x.shape[0], x.ctypes.data,
                                                            None if u is None else u.ctypes.data, 0))

    def ib_wss(self, normals, with_grad=False):
        """Wall shear stress at the Lagrangian points (Sec. 2.6) from the
        current velocity; normals (M, 3) unit outward.  Returns wss (M,) and,
        with with_grad, the velocity gradient (M, 3, 3), [p, i, j] = d u_i / d x_j."""
        M = self.ib_grid_info()["n_points"]
        n = np.ascontiguousarray(normals, dtype=np.float64).reshape(M, 3)
        w = np.empty(M)
        g = np.empty((M, 3, 3)) if with_grad else None
        self._check("ib_wss", self.lib.ib_wss(self.h, n.ctypes.data, w.ctypes.data,
                                              None if g is None else g.ctypes.data, 0))
        return (w, g) if with_grad else w

    def close(self):
        if getattr(self, "h", None):
            self.lib.ib_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class IBBatch:
    """Several deferred IBGrid problems stepped together (ib_batch_*)."""

    def __init__(self, members):
        self.lib = load_library()
        self.members = list(members)
        n = len(self.members)
        arr = (C.c_void_p * n)(*[m.h.value for m in self.members])
        h = C.c_void_p()
        s = self.lib.ib_batch_create(arr, n, C.byref(h))
        if s != 0:
            msg = self.members[0].lib.ib_last_error(self.members[0].h).decode() if n else ""
            raise IBError("ib_batch_create", s, msg)
        self.h = h

    def step(self, nsteps=1):
        """Advance every member; returns the per-member status of the last step."""
        st = np.zeros(len(self.members), dtype=np.int32)
        s = self.lib.ib_batch_step(self.h, int(nsteps), st.ctypes.data)
        if s not in (0, 4, 5):
            raise IBError("ib_batch_step", s, self.lib.ib_batch_last_error(self.h).decode())
        return st

    def info(self, i):
        info = _abi.IbInfo()
        s = self.lib.ib_batch_info(self.h, int(i), C.byref(info))
        if s != 0:
            raise IBError("ib_batch_info", s, "")
        return info.as_dict()

    def fields_get(self, i, field):
        return self.members[i].ib_fields_get(field)

    def close(self):
        if getattr(self, "h", None):
            self.lib.ib_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["IBGrid", "IBBatch", "IBError", "load_library", "FIELD"]
