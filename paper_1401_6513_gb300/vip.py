"""Thin ctypes binding of libvip (include/vip.h): argument marshalling only.

Every computation happens in the library's CUDA kernels.  Functions keep the C
names; array arguments accept numpy arrays (host memory) or any object with a
``data_ptr()`` (device or pinned host memory, e.g. torch tensors).  If the
library is missing the import fails with an error; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "libvip.so"

VIP_OK, VIP_ERR_ARG, VIP_ERR_CUDA, VIP_ERR_SINGULAR_STENCIL = 0, 1, 2, 3
VIP_ERR_NOT_CONVERGED, VIP_ERR_BREAKDOWN, VIP_ERR_NONFINITE, VIP_ERR_TIMEOUT, VIP_ERR_OOM = 4, 5, 6, 7, 8
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_SINGULAR_STENCIL",
                4: "ERR_NOT_CONVERGED", 5: "ERR_BREAKDOWN", 6: "ERR_NONFINITE",
                7: "ERR_TIMEOUT", 8: "ERR_OOM"}
VIP_NODE_INTERIOR, VIP_NODE_WALL, VIP_NODE_SLIP, VIP_NODE_OUTLET = 0, 1, 2, 3
VIP_W_CUBIC_SPLINE, VIP_W_PAPER = 0, 1
VIP_PREC_FP64, VIP_PREC_MIXED, VIP_PREC_MG32 = 0, 1, 2
VIP_IDENTITY_EXACT, VIP_IDENTITY_MLS = 0, 1
VIP_PROBES_NORMAL, VIP_PROBES_INSIDE = 0, 1
VIP_PRESSURE_INCREMENTAL, VIP_PRESSURE_KIM_MOIN, VIP_PRESSURE_INCREMENTAL_INTERIOR = 0, 1, 2
OPS = ["NBR", "D00", "D10", "D01", "D20", "D11", "D02", "LAPLACE", "VIP_E", "VIP_W", "VIP_N",
       "VIP_S", "GX", "GY", "HELM_U", "HELM_V", "POISSON"]
OP = {name: i for i, name in enumerate(OPS)}

# Every C entry point the header declares (checked by the CPU tests).
EXPORTS = ["vip_create", "vip_destroy", "vip_last_error", "vip_add_nodes", "vip_set_mls",
           "vip_set_flow", "vip_set_solver", "vip_build", "vip_set_state", "vip_step",
           "vip_get_state", "vip_get_stats", "vip_get_sizes", "vip_stencil_info",
           "vip_get_stencil", "vip_apply", "vip_convection", "vip_solve", "vip_load_state",
           "vip_set_profiling", "vip_get_profile", "vip_ws_collect", "vip_ws_train",
           "vip_ws_enable", "vip_ws_params", "vip_ws_eval", "vip_bicgstab_static",
           "vip_set_multigrid", "vip_autotune", "vip_get_geometry_iters", "vip_operator_layout",
           "vip_multigrid_info", "vip_set_mg_shift", "vip_set_refinement", "vip_checkpoint_size",
           "vip_checkpoint", "vip_ws_adam", "vip_ws_extrapolation", "vip_ws_set_loss",
           "vip_set_probes", "vip_set_pressure", "vip_set_inner_tolerance", "vip_ws_set_fit_window",
           "vip_3d_create", "vip_3d_destroy", "vip_3d_last_error", "vip_3d_set_nodes",
           "vip_3d_set_mls", "vip_3d_build", "vip_3d_stencil_size", "vip_3d_get_stencil",
           "vip_3d_apply", "vip_3d_set_flow", "vip_3d_set_state", "vip_3d_step",
           "vip_3d_get_state", "vip_3d_get_iters"]
OPS3 = ["NBR", "D000", "D100", "D010", "D001", "D200", "D020", "D002", "LAPLACE", "VIP_E", "VIP_W",
        "VIP_N", "VIP_S", "VIP_T", "VIP_B", "GX", "GY", "GZ", "NEUMANN"]
OP3 = {name: i for i, name in enumerate(OPS3)}
VIP_TUNE_MAX = 16
VIP_STATIC_MAX_ROWS = 131072
PHASES = ["rhs", "helmholtz", "divergence", "poisson", "project"]


class StepStats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("helm_iters", C.c_int32), ("poisson_iters", C.c_int32),
                ("poisson_outer", C.c_int32), ("status", C.c_int32), ("helm_relres", C.c_double),
                ("poisson_relres", C.c_double), ("total_poisson_iters", C.c_int64),
                ("total_poisson_outer", C.c_int64), ("total_helm_iters", C.c_int64)]


class TrainCfg(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("lr", C.c_double), ("seed", C.c_uint64),
                ("first_loss", C.c_double), ("final_loss", C.c_double), ("extrap", C.c_double),
                ("base_loss", C.c_double), ("net_kept", C.c_int32)]


class TuneResult(C.Structure):
    _fields_ = [("ncand", C.c_int32), ("best", C.c_int32), ("omega", C.c_float * VIP_TUNE_MAX),
                ("corr", C.c_float * VIP_TUNE_MAX), ("iters", C.c_int32 * VIP_TUNE_MAX),
                ("ms", C.c_double * VIP_TUNE_MAX)]

    def as_dict(self):
        n = self.ncand
        return {"omega": self.omega[self.best], "corr": self.corr[self.best],
                "candidates": [{"omega": round(self.omega[k], 4), "corr": round(self.corr[k], 4),
                                "iters": self.iters[k], "ms": round(self.ms[k], 3)} for k in range(n)]}


class VipError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib(path: str | Path | None = None):
    """Load libvip.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path else _LIB_PATH
    if not p.exists():
        raise ImportError(f"{p} is missing: build it with paper_1401_6513_gb300.build.build()")
    L = C.CDLL(str(p))
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "vip_create": ([C.POINTER(vp), C.c_int, vp], C.c_int),
        "vip_destroy": ([vp], None),
        "vip_last_error": ([vp], C.c_char_p),
        "vip_add_nodes": ([vp, i64, vp, vp, vp, vp, vp, vp, dbl, dbl, C.POINTER(i32)], C.c_int),
        "vip_set_mls": ([vp, C.c_int, C.c_int, dbl], C.c_int),
        "vip_set_flow": ([vp, i32, dbl, dbl], C.c_int),
        "vip_set_solver": ([vp, C.c_int, dbl, i32, C.c_int], C.c_int),
        "vip_set_refinement": ([vp, dbl], C.c_int),
        "vip_checkpoint_size": ([vp, C.POINTER(i64)], C.c_int),
        "vip_checkpoint": ([vp, C.c_int, vp], C.c_int),
        "vip_ws_adam": ([vp, dbl], C.c_int),
        "vip_ws_extrapolation": ([vp, C.c_int, C.POINTER(dbl)], C.c_int),
        "vip_ws_set_loss": ([vp, C.c_int, dbl], C.c_int),
        "vip_ws_set_fit_window": ([vp, i32], C.c_int),
        "vip_build": ([vp], C.c_int),
        "vip_set_state": ([vp, vp, vp, vp], C.c_int),
        "vip_step": ([vp, i32], C.c_int),
        "vip_get_state": ([vp, vp, vp, vp, vp], C.c_int),
        "vip_get_stats": ([vp, C.POINTER(StepStats)], C.c_int),
        "vip_get_sizes": ([vp, C.POINTER(i64), C.POINTER(i32)], C.c_int),
        "vip_stencil_info": ([vp, C.c_int, C.POINTER(i64), C.POINTER(i64)], C.c_int),
        "vip_get_stencil": ([vp, C.c_int, vp, vp, vp], C.c_int),
        "vip_apply": ([vp, C.c_int, vp, vp], C.c_int),
        "vip_convection": ([vp, vp, vp, vp, vp], C.c_int),
        "vip_solve": ([vp, C.c_int, vp, vp, C.c_int, dbl, i32, C.POINTER(i32), C.POINTER(dbl)],
                      C.c_int),
        "vip_load_state": ([vp, vp, vp, vp], C.c_int),
        "vip_set_profiling": ([vp, C.c_int], C.c_int),
        "vip_get_profile": ([vp, C.POINTER(dbl), C.POINTER(i64)], C.c_int),
        "vip_ws_collect": ([vp, C.c_int, i32], C.c_int),
        "vip_ws_train": ([vp, C.POINTER(TrainCfg)], C.c_int),
        "vip_ws_enable": ([vp, C.c_int], C.c_int),
        "vip_ws_params": ([vp, C.c_int, C.POINTER(C.c_float), C.POINTER(i64)], C.c_int),
        "vip_ws_eval": ([vp, i32, i32, vp, vp, vp, vp, vp, C.POINTER(dbl)], C.c_int),
        "vip_bicgstab_static": ([C.c_int, vp, i64, vp, vp, vp, vp, vp, dbl, i32, C.POINTER(i32),
                                 C.POINTER(dbl)], C.c_int),
        "vip_set_multigrid": ([vp, C.c_float, C.c_float], C.c_int),
        "vip_set_mg_shift": ([vp, i32, i32, i32], C.c_int),
        "vip_set_probes": ([vp, i32, C.c_int], C.c_int),
        "vip_set_pressure": ([vp, C.c_int], C.c_int),
        "vip_set_inner_tolerance": ([vp, C.c_int, C.c_double], C.c_int),
        "vip_get_geometry_iters": ([vp, vp], C.c_int),
        "vip_operator_layout": ([vp, C.c_int, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64),
                                 C.POINTER(i64)], C.c_int),
        "vip_multigrid_info": ([vp, C.POINTER(i32), C.POINTER(i64)], C.c_int),
        "vip_autotune": ([vp, C.POINTER(C.c_float), i32, C.POINTER(C.c_float), i32,
                          C.POINTER(TuneResult)], C.c_int),
        "vip_3d_create": ([C.POINTER(vp), C.c_int, vp], C.c_int),
        "vip_3d_destroy": ([vp], None),
        "vip_3d_last_error": ([vp], C.c_char_p),
        "vip_3d_set_nodes": ([vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, dbl, dbl, dbl], C.c_int),
        "vip_3d_set_mls": ([vp, C.c_int, dbl], C.c_int),
        "vip_3d_build": ([vp], C.c_int),
        "vip_3d_stencil_size": ([vp, C.c_int, C.POINTER(i64), C.POINTER(i64)], C.c_int),
        "vip_3d_get_stencil": ([vp, C.c_int, vp, vp, vp], C.c_int),
        "vip_3d_apply": ([vp, C.c_int, vp, vp], C.c_int),
        "vip_3d_set_flow": ([vp, dbl, dbl, dbl, i32], C.c_int),
        "vip_3d_set_state": ([vp, vp, vp, vp, vp], C.c_int),
        "vip_3d_step": ([vp, i32], C.c_int),
        "vip_3d_get_state": ([vp, vp, vp, vp, vp, vp], C.c_int),
        "vip_3d_get_iters": ([vp, C.POINTER(i64), C.POINTER(i32), C.POINTER(i32), C.POINTER(dbl)],
                             C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    if path is None:
        _lib = L
    return L


def _ptr(a):
    """Raw address of a numpy array or a tensor-like object (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _f64(a):
    if hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.float64)


class Build3D:
    """Owns one vip_3d handle (the 3D operator build); methods call the C entry
    points of the same name."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self.L = lib()
        h = C.c_void_p()
        st = self.L.vip_3d_create(C.byref(h), device, C.c_void_p(stream) if stream else None)
        self.h = h
        self._check(st)

    def _check(self, st):
        if st != VIP_OK:
            msg = self.L.vip_3d_last_error(self.h) if self.h else b"no handle"
            raise VipError(st, msg.decode() if msg else "")

    def close(self):
        if self.h:
            self.L.vip_3d_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vip_3d_set_nodes(self, x, y, z, kind, nx, ny, nz, h, Lx=0.0, Ly=0.0, Lz=0.0):
        x, y, z, nx, ny, nz, h = map(_f64, (x, y, z, nx, ny, nz, h))
        kind = kind if hasattr(kind, "data_ptr") else np.ascontiguousarray(kind, dtype=np.uint8)
        n = x.numel() if hasattr(x, "numel") else x.size
        self._check(self.L.vip_3d_set_nodes(self.h, n, _ptr(x), _ptr(y), _ptr(z), _ptr(kind),
                                            _ptr(nx), _ptr(ny), _ptr(nz), _ptr(h), Lx, Ly, Lz))

    def vip_3d_set_mls(self, weight=VIP_W_CUBIC_SPLINE, support=2.2):
        self._check(self.L.vip_3d_set_mls(self.h, weight, support))

    def vip_3d_build(self):
        self._check(self.L.vip_3d_build(self.h))

    def vip_3d_stencil_size(self, which):
        w = OP3[which] if isinstance(which, str) else int(which)
        nr, nz = C.c_int64(), C.c_int64()
        self._check(self.L.vip_3d_stencil_size(self.h, w, C.byref(nr), C.byref(nz)))
        return nr.value, nz.value

    def vip_3d_get_stencil(self, which):
        """Return (row_ptr, col, val) of a table as numpy arrays."""
        w = OP3[which] if isinstance(which, str) else int(which)
        nr, nz = self.vip_3d_stencil_size(w)
        ptr = np.empty(nr + 1, np.int64)
        col = np.empty(max(nz, 1), np.int32)
        val = np.empty(max(nz, 1), np.float64)
        self._check(self.L.vip_3d_get_stencil(self.h, w, _ptr(ptr), _ptr(col), _ptr(val)))
        return ptr, col[:nz], val[:nz]

    def vip_3d_apply(self, which, x, y=None):
        w = OP3[which] if isinstance(which, str) else int(which)
        x = _f64(x)
        if y is None:
            y = np.empty_like(x) if isinstance(x, np.ndarray) else None
        self._check(self.L.vip_3d_apply(self.h, w, _ptr(x), _ptr(y)))
        return y

    def vip_3d_set_flow(self, Re, dt, rtol=1e-8, max_iters=20000):
        self._check(self.L.vip_3d_set_flow(self.h, Re, dt, rtol, max_iters))

    def vip_3d_set_state(self, u, v, w, p):
        u, v, w, p = map(_f64, (u, v, w, p))
        self._check(self.L.vip_3d_set_state(self.h, _ptr(u), _ptr(v), _ptr(w), _ptr(p)))

    def vip_3d_step(self, nsteps=1):
        self._check(self.L.vip_3d_step(self.h, int(nsteps)))

    def vip_3d_get_state(self):
        """Return (u, v, w, p, phi) as numpy arrays."""
        nr, _ = self.vip_3d_stencil_size(0)
        out = [np.empty(nr, np.float64) for _ in range(5)]
        self._check(self.L.vip_3d_get_state(self.h, *(_ptr(a) for a in out)))
        return tuple(out)

    def vip_3d_get_iters(self):
        """(steps, Helmholtz iterations, Poisson iterations, Poisson relative residual)
        of the last step."""
        st, hi, pi, pr = C.c_int64(), C.c_int32(), C.c_int32(), C.c_double()
        self._check(self.L.vip_3d_get_iters(self.h, C.byref(st), C.byref(hi), C.byref(pi), C.byref(pr)))
        return st.value, hi.value, pi.value, pr.value


def build3d_for(ns, device=0, stream=None, weight=VIP_W_CUBIC_SPLINE, support=2.2) -> Build3D:
    """Create a 3D build handle for a NodeSet3-like object and build it."""
    b = Build3D(device, stream)
    b.vip_3d_set_mls(weight, support)
    b.vip_3d_set_nodes(ns.x, ns.y, ns.z, ns.kind, ns.nx, ns.ny, ns.nz, ns.h, ns.Lx, ns.Ly, ns.Lz)
    b.vip_3d_build()
    return b


class Context:
    """Owns one vip_ctx; methods call the C entry points of the same name."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self.L = lib()
        h = C.c_void_p()
        st = self.L.vip_create(C.byref(h), device, C.c_void_p(stream) if stream else None)
        self.h = h
        self._check(st)

    def _check(self, st):
        if st != VIP_OK:
            msg = self.L.vip_last_error(self.h)
            raise VipError(st, msg.decode() if msg else "")

    def close(self):
        if self.h:
            self.L.vip_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- setup -------------------------------------------------------------
    def vip_add_nodes(self, x, y, kind, nx, ny, h_local, Lx=0.0, Ly=0.0) -> int:
        x, y, nx, ny, h_local = map(_f64, (x, y, nx, ny, h_local))
        kind = kind if hasattr(kind, "data_ptr") else np.ascontiguousarray(kind, dtype=np.uint8)
        g = C.c_int32(-1)
        n = x.numel() if hasattr(x, "numel") else x.size
        self._check(self.L.vip_add_nodes(self.h, n, _ptr(x), _ptr(y), _ptr(kind), _ptr(nx),
                                         _ptr(ny), _ptr(h_local), float(Lx), float(Ly),
                                         C.byref(g)))
        return g.value

    def add_nodeset(self, ns) -> int:
        """Add a workloads.NodeSet and set its flow parameters."""
        g = self.vip_add_nodes(ns.x, ns.y, ns.kind, ns.nx, ns.ny, ns.h, ns.Lx, ns.Ly)
        self.vip_set_flow(g, ns.Re, ns.dt)
        return g

    def vip_set_mls(self, basis_order=2, weight=VIP_W_CUBIC_SPLINE, support=2.2):
        self._check(self.L.vip_set_mls(self.h, basis_order, weight, float(support)))

    def vip_set_flow(self, geom, Re, dt):
        self._check(self.L.vip_set_flow(self.h, int(geom), float(Re), float(dt)))

    def vip_set_solver(self, precision=VIP_PREC_FP64, rtol=1e-8, max_iters=20000,
                       identity=VIP_IDENTITY_EXACT):
        self._check(self.L.vip_set_solver(self.h, precision, float(rtol), int(max_iters), identity))

    def vip_set_refinement(self, inner_rtol=1e-4):
        self._check(self.L.vip_set_refinement(self.h, float(inner_rtol)))

    def vip_build(self):
        self._check(self.L.vip_build(self.h))

    # -- state and stepping --------------------------------------------------
    def vip_set_state(self, u, v, p=None):
        u, v = _f64(u), _f64(v)
        p = None if p is None else _f64(p)
        self._check(self.L.vip_set_state(self.h, _ptr(u), _ptr(v), _ptr(p)))

    def vip_load_state(self, u, v, p):
        self._check(self.L.vip_load_state(self.h, _ptr(u), _ptr(v), _ptr(p)))

    def vip_set_profiling(self, enable=True):
        self._check(self.L.vip_set_profiling(self.h, 1 if enable else 0))

    def vip_get_profile(self):
        ms = (C.c_double * 5)()
        n = C.c_int64()
        self._check(self.L.vip_get_profile(self.h, ms, C.byref(n)))
        return dict(zip(PHASES, list(ms))), n.value

    # -- learned warm start ------------------------------------------------------
    def vip_get_geometry_iters(self):
        """Poisson iterations of each geometry since vip_set_state (numpy int64)."""
        _, g = self.sizes()
        out = np.zeros(g, np.int64)
        self._check(self.L.vip_get_geometry_iters(self.h, _ptr(out)))
        return out

    def vip_set_multigrid(self, omega=1.0, corr=1.5):
        self._check(self.L.vip_set_multigrid(self.h, float(omega), float(corr)))

    def vip_set_mg_shift(self, geom, shift_x, shift_y):
        """Parity (0 or 1 per axis) of geometry geom's first multigrid cell grid
        (-1: every geometry); before vip_build."""
        self._check(self.L.vip_set_mg_shift(self.h, int(geom), int(shift_x), int(shift_y)))
        self.__dict__.setdefault("_mg_shift_calls", []).append((int(geom), int(shift_x), int(shift_y)))

    def vip_set_probes(self, geom, mode):
        """Normal-point placement VIP_PROBES_NORMAL / VIP_PROBES_INSIDE of geometry geom
        (-1: every geometry); before vip_build."""
        self._check(self.L.vip_set_probes(self.h, int(geom), int(mode)))
        self.__dict__.setdefault("_probe_calls", []).append((int(geom), int(mode)))

    def vip_set_inner_tolerance(self, which, inner_rtol):
        """Inner tolerance of the MIXED form's refinement for the solve `which`
        ("POISSON" or "HELM_U", the latter for both Helmholtz systems)."""
        self._check(self.L.vip_set_inner_tolerance(self.h, OP[which] if isinstance(which, str) else int(which),
                                                   float(inner_rtol)))

    def vip_set_pressure(self, form):
        """Pressure form VIP_PRESSURE_INCREMENTAL / _KIM_MOIN / _INCREMENTAL_INTERIOR."""
        self._check(self.L.vip_set_pressure(self.h, int(form)))

    def mg_shift_key(self):
        """The vip_set_mg_shift (and vip_set_probes) calls made on this context, as a
        suffix of the autotuning cache key ("" when both are the defaults everywhere)."""
        calls = self.__dict__.get("_mg_shift_calls", [])
        key = "|mg:" + ",".join(f"{g}:{x}{y}" for g, x, y in calls) if calls else ""
        probes = self.__dict__.get("_probe_calls", [])
        if any(m != VIP_PROBES_NORMAL for _, m in probes):
            key += "|probes:" + ",".join(f"{g}:{m}" for g, m in probes)
        return key

    def vip_autotune(self, omegas=(0.9, 1.0), corrs=(1.3, 1.5, 1.6, 1.7, 1.8, 1.9, 2.1)) -> TuneResult:
        """Time the last step's pressure-increment solve for every (omega, corr) pair
        and apply the fastest; returns the report."""
        om = (C.c_float * len(omegas))(*omegas)
        co = (C.c_float * len(corrs))(*corrs)
        res = TuneResult()
        self._check(self.L.vip_autotune(self.h, om, len(omegas), co, len(corrs), C.byref(res)))
        return res

    def vip_ws_collect(self, enable=True, max_samples=0):
        self._check(self.L.vip_ws_collect(self.h, 1 if enable else 0, int(max_samples)))

    def vip_ws_enable(self, enable=True):
        """enable: False/0 previous increment, True/1 extrapolation + network,
        2 extrapolation alone."""
        self._check(self.L.vip_ws_enable(self.h, int(enable)))

    def vip_ws_train(self, epochs=10, lr=1e-3, seed=0) -> TrainCfg:
        cfg = TrainCfg(epochs=int(epochs), lr=float(lr), seed=int(seed))
        self._check(self.L.vip_ws_train(self.h, C.byref(cfg)))
        return cfg

    def vip_ws_set_loss(self, kind=1, lam=0.01):
        """Network loss: 0 mean squared error, 1 residual proxy (lattice Laplacian)."""
        self._check(self.L.vip_ws_set_loss(self.h, int(kind), float(lam)))

    def vip_ws_set_fit_window(self, window=0):
        """Fit the extrapolation coefficient on the last `window` samples (0: all)."""
        self._check(self.L.vip_ws_set_fit_window(self.h, int(window)))

    def vip_ws_extrapolation(self, a=None):
        """Read the warm start's extrapolation coefficient, or set it to a."""
        v = C.c_double(0.0 if a is None else float(a))
        self._check(self.L.vip_ws_extrapolation(self.h, 0 if a is None else 1, C.byref(v)))
        return v.value

    def vip_ws_adam(self, lr=1e-3):
        self._check(self.L.vip_ws_adam(self.h, float(lr)))

    def vip_ws_params(self, params=None):
        """Return the FP32 parameters; with `params`, load them instead."""
        n = C.c_int64()
        self._check(self.L.vip_ws_params(self.h, 0, None, C.byref(n)))
        if params is None:
            out = np.empty(n.value, np.float32)
            self._check(self.L.vip_ws_params(self.h, 0, out.ctypes.data_as(C.POINTER(C.c_float)), None))
            return out
        buf = np.ascontiguousarray(params, np.float32)
        assert buf.size == n.value
        self._check(self.L.vip_ws_params(self.h, 1, buf.ctypes.data_as(C.POINTER(C.c_float)), None))
        return buf

    def vip_step(self, nsteps=1):
        self._check(self.L.vip_step(self.h, int(nsteps)))

    def vip_get_state(self, u=None, v=None, p=None, phi=None):
        """Fill the given buffers; with no buffers, return fresh numpy arrays."""
        if u is None and v is None and p is None and phi is None:
            n = self.sizes()[0]
            u, v, p, phi = (np.empty(n) for _ in range(4))
        self._check(self.L.vip_get_state(self.h, _ptr(u), _ptr(v), _ptr(p), _ptr(phi)))
        return u, v, p, phi

    def vip_checkpoint_size(self) -> int:
        n = C.c_int64()
        self._check(self.L.vip_checkpoint_size(self.h, C.byref(n)))
        return n.value

    def vip_checkpoint(self, save, buf=None):
        """save=True: write a checkpoint into buf (a uint8 numpy array or a tensor of
        vip_checkpoint_size() bytes; allocated on the host if None) and return it;
        save=False: restore the checkpoint held in buf."""
        if buf is None:
            if not save:
                raise ValueError("restoring needs a buffer")
            buf = np.zeros(self.vip_checkpoint_size(), np.uint8)
        ptr = buf.data_ptr() if hasattr(buf, "data_ptr") else buf.ctypes.data
        self._check(self.L.vip_checkpoint(self.h, 1 if save else 0, C.c_void_p(ptr)))
        return buf

    def vip_get_stats(self) -> StepStats:
        s = StepStats()
        self._check(self.L.vip_get_stats(self.h, C.byref(s)))
        return s

    def sizes(self):
        n = C.c_int64()
        g = C.c_int32()
        self._check(self.L.vip_get_sizes(self.h, C.byref(n), C.byref(g)))
        return n.value, g.value

    # -- inspection ----------------------------------------------------------
    def vip_operator_layout(self, which):
        """Device storage of a Krylov operator: dict with slices, uniform_slices,
        uniform_entries and other_entries (see the C header)."""
        w = OP[which] if isinstance(which, str) else int(which)
        v = [C.c_int64() for _ in range(4)]
        self._check(self.L.vip_operator_layout(self.h, w, *(C.byref(x) for x in v)))
        return dict(zip(("slices", "uniform_slices", "uniform_entries", "other_entries"),
                        (x.value for x in v)))

    def vip_multigrid_info(self):
        """(coarse levels, entries of the dense coarsest inverses) of the Poisson
        preconditioner."""
        lv, ce = C.c_int32(), C.c_int64()
        self._check(self.L.vip_multigrid_info(self.h, C.byref(lv), C.byref(ce)))
        return lv.value, ce.value

    def vip_get_stencil(self, which):
        """Return (row_ptr, col, val) of a table as numpy arrays."""
        w = OP[which] if isinstance(which, str) else int(which)
        nr, nz = C.c_int64(), C.c_int64()
        self._check(self.L.vip_stencil_info(self.h, w, C.byref(nr), C.byref(nz)))
        ptr = np.empty(nr.value + 1, np.int64)
        col = np.empty(max(nz.value, 1), np.int32)
        val = np.empty(max(nz.value, 1), np.float64)
        self._check(self.L.vip_get_stencil(self.h, w, _ptr(ptr), _ptr(col), _ptr(val)))
        return ptr, col[:nz.value], val[:nz.value]

    def vip_apply(self, which, x, y=None):
        w = OP[which] if isinstance(which, str) else int(which)
        x = _f64(x)
        if y is None:
            y = np.empty_like(x) if isinstance(x, np.ndarray) else None
        self._check(self.L.vip_apply(self.h, w, _ptr(x), _ptr(y)))
        return y

    def vip_convection(self, u, v):
        u, v = _f64(u), _f64(v)
        Nu, Nv = np.empty_like(u), np.empty_like(v)
        self._check(self.L.vip_convection(self.h, _ptr(u), _ptr(v), _ptr(Nu), _ptr(Nv)))
        return Nu, Nv

    def vip_solve(self, which, b, x0, precision=VIP_PREC_FP64, rtol=1e-8, max_iters=20000):
        w = OP[which] if isinstance(which, str) else int(which)
        b = _f64(b)
        x = np.array(x0, dtype=np.float64, copy=True)
        it = C.c_int32()
        rr = C.c_double()
        self._check(self.L.vip_solve(self.h, w, _ptr(b), _ptr(x), precision, float(rtol),
                                     int(max_iters), C.byref(it), C.byref(rr)))
        return x, it.value, rr.value


def vip_bicgstab_static(device, stream, n, row_ptr, col, val, b, x, rtol=1e-10, max_iters=20000):
    """FP64 BiCGSTAB on a caller-owned device CSR matrix without any device
    allocation (workspace in static device memory, n <= VIP_STATIC_MAX_ROWS).
    All arrays are device tensors; x is the initial guess and is overwritten.
    Returns (status, iterations, true relative residual)."""
    it, rr = C.c_int32(0), C.c_double(0.0)
    st = lib().vip_bicgstab_static(int(device), C.c_void_p(stream) if stream else None, int(n),
                                   _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(b), _ptr(x),
                                   float(rtol), int(max_iters), C.byref(it), C.byref(rr))
    return st, it.value, rr.value


MG_SHIFTS = ((0, 0), (1, 0), (0, 1), (1, 1))


def choose_mg_shifts(nodesets, steps=2, make=None, **solver_kw):
    """Cell-grid parity of the multigrid for every node set: one context per parity
    in MG_SHIFTS (all node sets in it, a periodic axis kept at 0), `steps` steps
    from the initial state, and for each node set the parity whose Poisson solves
    took the fewest iterations (vip_get_geometry_iters).  A context whose steps fail
    counts as the worst for all its node sets.  Returns (shifts, iterations [4, G])."""
    if not isinstance(nodesets, (list, tuple)):
        nodesets = [nodesets]
    make = make or solver_for
    its = np.full((len(MG_SHIFTS), len(nodesets)), np.iinfo(np.int64).max, np.int64)
    seen = {}
    for k, (sx, sy) in enumerate(MG_SHIFTS):
        shifts = [(0 if ns.Lx > 0 else sx, 0 if ns.Ly > 0 else sy) for ns in nodesets]
        if tuple(shifts) in seen:  # periodic axes make some parities coincide
            its[k] = its[seen[tuple(shifts)]]
            continue
        seen[tuple(shifts)] = k
        ctx = make(nodesets, mg_shifts=shifts, **solver_kw)
        try:
            ctx.vip_step(steps)
            its[k] = ctx.vip_get_geometry_iters()
        except VipError:
            pass
        finally:
            ctx.close()
    best = its.argmin(axis=0)
    return [(0 if ns.Lx > 0 else MG_SHIFTS[b][0], 0 if ns.Ly > 0 else MG_SHIFTS[b][1])
            for ns, b in zip(nodesets, best)], its


PREC_NAMES = {VIP_PREC_FP64: "fp64", VIP_PREC_MIXED: "mixed", VIP_PREC_MG32: "mg32"}


def choose_precision(ctx, candidates=(VIP_PREC_MIXED, VIP_PREC_FP64), steps=2, rtol=1e-8,
                     max_iters=50000, identity=VIP_IDENTITY_EXACT):
    """Precision form of the Krylov solves chosen by measurement: from one checkpoint of
    the context's current state, every form in `candidates` takes one untimed step
    (its step graph is captured) and then, again from the checkpoint, `steps` steps
    whose device time is the sum of the step phases' CUDA-event times
    (vip_set_profiling).  A form whose steps fail (any device status) is left out.
    The fastest form is set on the context and the state restored, so the caller
    continues from where it was.  Every form stops its solves on the same FP64
    residual, so the choice changes cost, not the tolerance.  Returns (precision,
    table of {precision, ms, poisson_iters, error})."""
    ck = ctx.vip_checkpoint(True)
    table, times = [], {}
    for prec in candidates:
        rec = {"precision": PREC_NAMES.get(prec, prec), "ms": None}
        try:
            ctx.vip_set_solver(prec, rtol, max_iters, identity)
            ctx.vip_checkpoint(False, ck)
            ctx.vip_step(1)
            ctx.vip_checkpoint(False, ck)
            s0 = ctx.vip_get_stats()
            ctx.vip_set_profiling(True)
            try:
                ctx.vip_step(steps)
                s1 = ctx.vip_get_stats()
                phase_ms, n = ctx.vip_get_profile()
            finally:
                ctx.vip_set_profiling(False)
            rec["ms"] = sum(phase_ms.values()) / max(n, 1)
            rec["poisson_iters"] = (s1.total_poisson_iters - s0.total_poisson_iters) / steps
            times[prec] = rec["ms"]
        except VipError as e:
            rec["error"] = str(e)
        table.append(rec)
    if not times:
        ctx.vip_checkpoint(False, ck)
        raise VipError(VIP_ERR_NOT_CONVERGED, "choose_precision: no form completed its steps")
    best = min(times, key=times.get)
    ctx.vip_set_solver(best, rtol, max_iters, identity)
    ctx.vip_checkpoint(False, ck)
    return best, table


def geometry_signature(nodesets) -> str:
    """Key of a set of node sets for the autotuning cache: names, node counts and a
    hash of the coordinates and kinds."""
    import hashlib
    hsh = hashlib.sha1()
    parts = []
    for ns in nodesets:
        parts.append(f"{ns.name}:{ns.n}")
        hsh.update(np.ascontiguousarray(ns.x, dtype=np.float64).tobytes())
        hsh.update(np.ascontiguousarray(ns.y, dtype=np.float64).tobytes())
        hsh.update(np.ascontiguousarray(ns.kind, dtype=np.uint8).tobytes())
    return "|".join(parts) + "|" + hsh.hexdigest()[:16]


def autotune(ctx, nodesets, cache=None, omegas=(0.9, 1.0), corrs=(1.3, 1.5, 1.6, 1.7, 1.8, 1.9, 2.1),
             refine=3, refine_steps=3):
    """Pick the multigrid parameters of a context built from `nodesets`: from the JSON
    file `cache` when it has this geometry signature (with the context's cell-grid
    parities), else in two stages, then store
    the choice there:
      1. vip_autotune after one step: every (omega, corr) pair solves that step's
         pressure-increment system from a zero guess, timed on the device;
      2. the `refine` fastest pairs each run `refine_steps` steps from the node sets'
         initial fields, scored by the Poisson iterations of the steps after the first
         (warm-started like the steps that follow; the cost of an iteration does not
         depend on the pair, so iterations rank them without timing noise).
    The state is reset to the initial fields afterwards.  Returns the chosen
    {"omega", "corr", ...} entry."""
    import json
    # the hierarchy, hence the best parameters, depends on the cell-grid parity too
    key = geometry_signature(nodesets) + getattr(ctx, "mg_shift_key", lambda: "")()
    table = {}
    if cache is not None and Path(cache).exists():
        table = json.loads(Path(cache).read_text())
    if key in table:
        entry = table[key]
        ctx.vip_set_multigrid(entry["omega"], entry["corr"])
        return dict(entry, cached=True)

    def reset():
        ctx.vip_set_state(np.concatenate([ns.u0 for ns in nodesets]),
                          np.concatenate([ns.v0 for ns in nodesets]),
                          np.concatenate([ns.p0 for ns in nodesets]))

    ctx.vip_step(1)
    entry = ctx.vip_autotune(omegas, corrs).as_dict()
    cands = sorted((c for c in entry["candidates"] if c["ms"] >= 0), key=lambda c: c["ms"])[:refine]
    if refine_steps > 1 and len(cands) > 1:
        scored = []
        for c in cands:
            ctx.vip_set_multigrid(c["omega"], c["corr"])
            reset()
            ctx.vip_step(1)
            i0 = ctx.vip_get_stats().total_poisson_iters
            ctx.vip_step(refine_steps - 1)
            c["step_iters"] = ctx.vip_get_stats().total_poisson_iters - i0
            scored.append(c)
        best = min(scored, key=lambda c: (c["step_iters"], c["ms"]))
        entry["omega"], entry["corr"] = best["omega"], best["corr"]
        entry["refined_on_steps"] = refine_steps - 1
    ctx.vip_set_multigrid(entry["omega"], entry["corr"])
    reset()
    if cache is not None:
        table[key] = entry
        Path(cache).parent.mkdir(parents=True, exist_ok=True)
        Path(cache).write_text(json.dumps(table, indent=1))
    return dict(entry, cached=False)


def solver_for(nodesets, precision=VIP_PREC_FP64, rtol=1e-8, max_iters=20000,
               identity=VIP_IDENTITY_EXACT, weight=VIP_W_CUBIC_SPLINE, support=2.2,
               device=0, stream=None, set_state=True, mg_shifts=None, probes="normal",
               pressure="incremental") -> Context:
    """Create a context for one node set or a list of them, build it and set u0, v0, p0.
    mg_shifts: one (shift_x, shift_y) per node set for vip_set_mg_shift (default 0, 0).
    probes: "normal" or "inside", the normal-point placement of every node set
    (vip_set_probes).  pressure: "incremental", "kim_moin" or "incremental_interior"
    (vip_set_pressure)."""
    if not isinstance(nodesets, (list, tuple)):
        nodesets = [nodesets]
    ctx = Context(device, stream)
    for ns in nodesets:
        ctx.add_nodeset(ns)
    if mg_shifts is not None:
        if len(mg_shifts) != len(nodesets):
            raise ValueError("one (shift_x, shift_y) per node set")
        for g, (sx, sy) in enumerate(mg_shifts):
            ctx.vip_set_mg_shift(g, sx, sy)
    modes = {"normal": VIP_PROBES_NORMAL, "inside": VIP_PROBES_INSIDE}
    if probes not in modes:
        raise ValueError(f"probes must be 'normal' or 'inside', not {probes!r}")
    if probes != "normal":
        ctx.vip_set_probes(-1, modes[probes])
    forms = {"incremental": VIP_PRESSURE_INCREMENTAL, "kim_moin": VIP_PRESSURE_KIM_MOIN,
             "incremental_interior": VIP_PRESSURE_INCREMENTAL_INTERIOR}
    if pressure not in forms:
        raise ValueError(f"pressure must be one of {sorted(forms)}, not {pressure!r}")
    if pressure != "incremental":
        ctx.vip_set_pressure(forms[pressure])
    ctx.vip_set_mls(2, weight, support)
    ctx.vip_set_solver(precision, rtol, max_iters, identity)
    ctx.vip_build()
    if set_state:
        ctx.vip_set_state(np.concatenate([ns.u0 for ns in nodesets]),
                          np.concatenate([ns.v0 for ns in nodesets]),
                          np.concatenate([ns.p0 for ns in nodesets]))
    return ctx
