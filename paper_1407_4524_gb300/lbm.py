"""Thin Python binding of liblbm (include/lbm.h): argument marshalling only.

Every step of the lattice-Boltzmann path runs in the CUDA kernels of
liblbm.so; this module converts a problem-description dict (see
``workloads``) into the C descriptor, optionally routes the library's device
allocations through PyTorch's caching allocator and enqueues on a PyTorch
stream.  There is no CPU fallback: if the library is missing or no GPU is
present, construction raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

LBM_OK = 0
ERRORS = {1: "LBM_ERR_ARG", 2: "LBM_ERR_OOM", 3: "LBM_ERR_CUDA", 4: "LBM_ERR_UNSTABLE",
          5: "LBM_ERR_TIMEOUT", 6: "LBM_ERR_STATE"}
PRECISION = {"fp64": 0, "fp32": 1, "fp16": 2}
EDGE = {"periodic": 0, "wall": 1, "inlet": 2, "outlet": 3}
SHAPE = {"cylinder": 0, "sphere": 1, "ellipse": 2}
FT_KIND = {"static": 0, "lattice": 1, "moving": 2, "impulsive": 3}
SERIES_ROW = 18

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class lbm_domain_desc(C.Structure):
    _fields_ = [
        ("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("precision", C.c_int), ("equilibrium", C.c_int), ("edge", C.c_int * 6),
        ("inlet_profile", C.c_int), ("refill", C.c_int), ("has_force", C.c_int),
        ("device", C.c_int), ("tau", C.c_double), ("rho0", C.c_double), ("u_in", C.c_double),
        ("force", C.c_double * 3), ("u0", C.c_double * 3), ("series_capacity", C.c_int64),
        ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p),
        ("gravity", C.c_double * 3), ("edge_rule", C.c_int), ("free_scheme", C.c_int),
    ]


class lbm_body(C.Structure):
    _fields_ = [
        ("shape", C.c_int), ("halfway", C.c_int), ("free_body", C.c_int), ("reserved", C.c_int),
        ("R", C.c_double), ("X0", C.c_double * 3), ("U", C.c_double * 3), ("W", C.c_double * 3),
        ("t0", C.c_int64), ("density_ratio", C.c_double), ("R2", C.c_double), ("theta0", C.c_double),
    ]


class lbm_batch_desc(C.Structure):
    _fields_ = [
        ("device", C.c_int), ("max_slots", C.c_int), ("ticks_per_launch", C.c_int), ("reserved", C.c_int),
        ("budget_bytes", C.c_int64), ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
        ("alloc_ctx", C.c_void_p),
    ]


class lbm_stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("step", "cells", "fluid_cells", "links", "fallback_links",
                                          "covered", "uncovered", "device_bytes", "h2d_bytes", "d2h_bytes",
                                          "timeouts", "unstable", "extrapolated")]


class LbmError(RuntimeError):
    pass


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblbm.so (building it first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise LbmError(f"liblbm.so not found at {path}; run paper_1407_4524_gb300/build.py")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.lbm_last_error.restype = C.c_char_p
    lib.lbm_version.restype = C.c_char_p
    lib.lbm_lattice_table.argtypes = [C.c_int, P, P, P]
    lib.lbm_create_domain.argtypes = [C.POINTER(lbm_domain_desc), C.POINTER(C.c_void_p)]
    lib.lbm_destroy_domain.argtypes = [P]
    lib.lbm_set_bodies.argtypes = [P, C.POINTER(lbm_body), C.c_int]
    lib.lbm_update_bodies.argtypes = [P, C.POINTER(lbm_body), C.c_int]
    lib.lbm_step.argtypes = [P, C.c_int]
    lib.lbm_prepare_graph.argtypes = [P]
    lib.lbm_get_force_torque.argtypes = [P, C.c_int64, C.c_int64, C.c_int, P]
    lib.lbm_get_series.argtypes = [P, C.c_int64, C.c_int64, P]
    lib.lbm_get_populations.argtypes = [P, P]
    lib.lbm_set_populations.argtypes = [P, P]
    lib.lbm_get_macros.argtypes = [P, P]
    lib.lbm_state_bytes.restype = C.c_int64
    lib.lbm_state_bytes.argtypes = [P]
    lib.lbm_save_state.argtypes = [P, P, C.c_int64]
    lib.lbm_load_state.argtypes = [P, P, C.c_int64]
    lib.lbm_get_solid.argtypes = [P, P]
    lib.lbm_get_body_state.argtypes = [P, P]
    lib.lbm_get_stats.argtypes = [P, C.POINTER(lbm_stats)]
    lib.lbm_time.restype = C.c_int64
    lib.lbm_time.argtypes = [P]
    lib.lbm_set_stream.argtypes = [P, P]
    lib.lbm_set_kernel_timing.argtypes = [P, C.c_int]
    lib.lbm_kernel_time.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_double)]
    lib.lbm_launches_per_step.argtypes = [P, C.POINTER(C.c_int)]
    lib.lbm_batch_create.argtypes = [C.POINTER(lbm_batch_desc), C.POINTER(C.c_void_p)]
    lib.lbm_batch_destroy.argtypes = [P]
    lib.lbm_batch_solve_bytes.argtypes = [C.POINTER(lbm_domain_desc), C.POINTER(lbm_body), C.c_int, C.c_int64,
                                          C.POINTER(C.c_int64)]
    lib.lbm_batch_admit.argtypes = [P, C.POINTER(lbm_domain_desc), C.POINTER(lbm_body), C.c_int, C.c_int64,
                                    C.POINTER(C.c_int)]
    lib.lbm_batch_run.argtypes = [P, C.c_int]
    lib.lbm_batch_poll.argtypes = [P, P, C.c_int, C.POINTER(C.c_int)]
    lib.lbm_batch_get_force_torque.argtypes = [P, C.c_int, C.c_int64, C.c_int64, C.c_int, P]
    lib.lbm_batch_time.restype = C.c_int64
    lib.lbm_batch_time.argtypes = [P, C.c_int]
    lib.lbm_batch_release.argtypes = [P, C.c_int]
    lib.lbm_batch_usage.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int64)]
    _lib = lib
    return lib


def _check(rc: int):
    if rc != LBM_OK:
        msg = _lib.lbm_last_error().decode(errors="replace")
        raise LbmError(f"{ERRORS.get(rc, rc)}: {msg}")


def lbm_lattice_table(q: int):
    """(c[Q,3], w[Q], opp[Q]) in the library's direction order; needs no GPU."""
    lib = load()
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    opp = np.zeros(q, dtype=np.int32)
    _check(lib.lbm_lattice_table(q, c.ctypes.data, w.ctypes.data, opp.ctypes.data))
    return c, w, opp


def body_struct(b: dict) -> lbm_body:
    s = lbm_body()
    s.shape = SHAPE[b.get("shape", "sphere")]
    s.halfway = int(bool(b.get("halfway", False)))
    s.R = float(b["R"])
    X0 = tuple(b["X0"]) + (0.0,) * (3 - len(b["X0"]))
    U = tuple(b.get("U", (0.0, 0.0, 0.0)))
    U = U + (0.0,) * (3 - len(U))
    W = b.get("W", (0.0, 0.0, 0.0))
    if np.isscalar(W):
        W = (0.0, 0.0, float(W))
    for k in range(3):
        s.X0[k], s.U[k], s.W[k] = float(X0[k]), float(U[k]), float(W[k])
    s.t0 = int(b.get("t0", 0))
    s.free_body = int(bool(b.get("free", False)))
    s.density_ratio = float(b.get("density_ratio", 1.0))
    s.R2 = float(b.get("R2", b["R"]))
    s.theta0 = float(b.get("theta0", 0.0))
    return s


def domain_desc(spec: dict, device: int = 0, series_capacity: int = 0):
    """(lbm_domain_desc, Q, (nx, ny, nz)) of a problem dict; stream and
    allocator are left unset."""
    q = {"D2Q9": 9, "D3Q19": 19}[spec["lattice"]]
    n = tuple(spec["n"]) + (1,) * (3 - len(spec["n"]))
    d = lbm_domain_desc()
    d.lattice, d.nx, d.ny, d.nz = q, n[0], n[1], n[2]
    d.precision = PRECISION[spec.get("precision", "fp32")]
    d.equilibrium = {"incomp": 0, "standard": 1}[spec.get("eq", "incomp")]
    edges = spec.get("edges", {})
    k = 0
    for ax in "xyz":
        e = edges.get(ax, "periodic")
        lo, hi = (e, e) if isinstance(e, str) else e
        d.edge[k], d.edge[k + 1] = EDGE[lo], EDGE[hi]
        k += 2
    inlet = spec.get("inlet", {})
    d.inlet_profile = 1 if inlet.get("profile", "uniform") == "parabolic" else 0
    d.u_in = float(inlet.get("u", 0.0))
    d.refill = {"uB": 0, "ubar": 1, "extrap": 2}[spec.get("refill", "uB")]
    d.edge_rule = {"link": 0, "zouhe": 1}[spec.get("edge_rule", "link")]
    d.free_scheme = {"explicit": 0, "aidun": 1, "predictor": 2}[spec.get("free_scheme", "explicit")]
    g = spec.get("force")
    d.has_force = int(g is not None)
    for j in range(3):
        d.force[j] = float(g[j]) if g is not None and j < len(g) else 0.0
    u0 = tuple(spec.get("u0", (0.0, 0.0, 0.0)))
    for j in range(3):
        d.u0[j] = float(u0[j]) if j < len(u0) else 0.0
    d.tau = float(spec["tau"])
    d.rho0 = float(spec.get("rho0", 1.0))
    gv = tuple(spec.get("gravity", (0.0, 0.0, 0.0)))
    for j in range(3):
        d.gravity[j] = float(gv[j]) if j < len(gv) else 0.0
    d.device = int(device)
    d.series_capacity = int(series_capacity or spec.get("series_capacity", 0) or 0)
    return d, q, n


def body_array(bodies):
    return (lbm_body * max(len(bodies), 1))(*[body_struct(b) for b in bodies])


class _TorchAllocator:
    """Routes the library's device allocations through torch's caching allocator."""

    def __init__(self, device: int, stream_ptr: int):
        import torch
        self.torch = torch
        self.device = device
        self.stream_ptr = stream_ptr

        def _alloc(nbytes, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                              self.stream_ptr or None))
            except Exception:  # OOM -> the library reports LBM_ERR_OOM
                return None

        def _free(ptr, ctx):
            if ptr:
                torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


class Domain:
    """One lattice-Boltzmann domain on the GPU, built from a problem dict."""

    def __init__(self, spec: dict, device: int = 0, stream=None, torch_allocator: bool = True,
                 series_capacity: int = 0):
        lib = load()
        self.lib = lib
        self.spec = spec
        d, q, n = domain_desc(spec, device, series_capacity)
        self._alloc = None
        self.stream = stream
        stream_ptr = 0
        try:
            import torch
            if torch.cuda.is_available():
                if stream is None:
                    stream = torch.cuda.current_stream(device)
                    self.stream = stream
                stream_ptr = int(stream.cuda_stream)
                if torch_allocator:
                    self._alloc = _TorchAllocator(device, stream_ptr)
        except ImportError:
            pass
        d.stream = C.c_void_p(stream_ptr) if stream_ptr else None
        if self._alloc is not None:
            d.alloc, d.free = self._alloc.alloc, self._alloc.free
        self._desc = d
        h = C.c_void_p()
        _check(lib.lbm_create_domain(C.byref(d), C.byref(h)))
        self.h = h
        self.q, self.shape = q, n
        self.N = n[0] * n[1] * n[2]
        self.bodies = list(spec.get("bodies", []))
        if self.bodies:
            self.set_bodies(self.bodies)

    # ------------------------------------------------------------ lifecycle --
    def close(self):
        if getattr(self, "h", None):
            self.lib.lbm_destroy_domain(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_bodies(self, bodies):
        arr = (lbm_body * max(len(bodies), 1))(*[body_struct(b) for b in bodies])
        _check(self.lib.lbm_set_bodies(self.h, arr, len(bodies)))
        self.bodies = list(bodies)

    def update_bodies(self, bodies):
        arr = (lbm_body * len(bodies))(*[body_struct(b) for b in bodies])
        _check(self.lib.lbm_update_bodies(self.h, arr, len(bodies)))
        self.bodies = list(bodies)

    def step(self, n: int = 1):
        _check(self.lib.lbm_step(self.h, int(n)))

    def prepare_graph(self):
        """record the 16-step graph now (lbm_prepare_graph): later runs of
        >= 16 steps replay it without the recording cost"""
        _check(self.lib.lbm_prepare_graph(self.h))

    @property
    def t(self) -> int:
        return int(self.lib.lbm_time(self.h))

    # -------------------------------------------------------------- results --
    def series(self, first: int = 0, count: int | None = None) -> np.ndarray:
        nb = len(self.bodies)
        if count is None:
            count = self.t - first
        out = np.zeros((count, max(nb, 1), SERIES_ROW))
        if nb and count:
            _check(self.lib.lbm_get_series(self.h, first, count, out.ctypes.data))
        return out[:, :nb]

    def force_torque(self, kind: str = "static", first: int = 0, count: int | None = None) -> np.ndarray:
        nb = len(self.bodies)
        if count is None:
            count = self.t - first
        out = np.zeros((count, max(nb, 1), 6))
        if nb and count:
            _check(self.lib.lbm_get_force_torque(self.h, first, count, FT_KIND[kind], out.ctypes.data))
        return out[:, :nb]

    def populations(self) -> np.ndarray:
        """post-collision f-hat(t) as FP64 f, shape [Q, nz, ny, nx]"""
        out = np.empty(self.q * self.N)
        _check(self.lib.lbm_get_populations(self.h, out.ctypes.data))
        nx, ny, nz = self.shape
        return out.reshape(self.q, nz, ny, nx)

    def set_populations(self, f: np.ndarray):
        """set f(t) (pre-collision, FP64, shape [Q, nz, ny, nx] or [Q, N]); the
        library collides it into the state the next step starts from"""
        a = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(self.q, self.N))
        _check(self.lib.lbm_set_populations(self.h, a.ctypes.data))

    def macros(self) -> np.ndarray:
        """rho, u_x, u_y, u_z at t, shape [4, nz, ny, nx] (zero at solid nodes)"""
        out = np.empty(4 * self.N)
        _check(self.lib.lbm_get_macros(self.h, out.ctypes.data))
        nx, ny, nz = self.shape
        return out.reshape(4, nz, ny, nx)

    def save_state(self) -> bytes:
        """snapshot of the whole state at the current step (checkpoint)"""
        n = int(self.lib.lbm_state_bytes(self.h))
        buf = np.empty(n, dtype=np.uint8)
        _check(self.lib.lbm_save_state(self.h, buf.ctypes.data, n))
        return buf.tobytes()

    def load_state(self, blob: bytes):
        """restore a snapshot taken from a domain of the same problem (resume)"""
        buf = np.frombuffer(blob, dtype=np.uint8)
        _check(self.lib.lbm_load_state(self.h, buf.ctypes.data, len(buf)))

    def body_state(self) -> np.ndarray:
        """[n_bodies, 9]: X(t), U(t), W(t)"""
        nb = len(self.bodies)
        out = np.zeros(max(nb, 1) * 9)
        if nb:
            _check(self.lib.lbm_get_body_state(self.h, out.ctypes.data))
        return out.reshape(-1, 9)[:nb]

    def solid(self) -> np.ndarray:
        out = np.empty(self.N, dtype=np.int32)
        _check(self.lib.lbm_get_solid(self.h, out.ctypes.data))
        nx, ny, nz = self.shape
        return out.reshape(nz, ny, nx)

    def stats(self) -> dict:
        s = lbm_stats()
        _check(self.lib.lbm_get_stats(self.h, C.byref(s)))
        return {k: int(getattr(s, k)) for k, _ in lbm_stats._fields_}

    # --------------------------------------------------------------- timing --
    def set_kernel_timing(self, enable: bool):
        _check(self.lib.lbm_set_kernel_timing(self.h, int(bool(enable))))

    def kernel_time(self):
        n = C.c_int64()
        ms = C.c_double()
        _check(self.lib.lbm_kernel_time(self.h, C.byref(n), C.byref(ms)))
        return int(n.value), float(ms.value)

    def launches_per_step(self) -> int:
        v = C.c_int()
        _check(self.lib.lbm_launches_per_step(self.h, C.byref(v)))
        return int(v.value)


class Batch:
    """A serving batch (include/lbm.h, lbm_batch_*): many static-body solves in
    the reduced-precision modes resident on one GPU, admitted against a
    device-memory budget and advanced together, ``ticks_per_launch`` steps per
    replay of the batch's tick graph."""

    def __init__(self, budget_bytes: int, max_slots: int = 64, ticks_per_launch: int = 32, device: int = 0,
                 torch_allocator: bool = True):
        lib = load()
        self.lib = lib
        import torch
        if not torch.cuda.is_available():
            raise LbmError("a serving batch needs a CUDA device")
        self.device = int(device)
        # a stream of its own: the tick graph is captured on it (the legacy
        # default stream cannot be captured)
        self.stream = torch.cuda.Stream(device)
        stream_ptr = int(self.stream.cuda_stream)
        d = lbm_batch_desc()
        d.device, d.max_slots, d.ticks_per_launch = self.device, int(max_slots), int(ticks_per_launch)
        d.budget_bytes = int(budget_bytes)
        d.stream = C.c_void_p(stream_ptr)
        self._alloc = _TorchAllocator(self.device, stream_ptr) if torch_allocator else None
        if self._alloc is not None:
            d.alloc, d.free = self._alloc.alloc, self._alloc.free
        self._desc = d
        h = C.c_void_p()
        _check(lib.lbm_batch_create(C.byref(d), C.byref(h)))
        self.h = h
        self.ticks_per_launch = int(ticks_per_launch) or 32
        self.specs = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _steps(spec, steps):
        return int(spec["steps"] if steps is None else steps)

    def solve_bytes(self, spec: dict, steps: int | None = None) -> int:
        d, _, _ = domain_desc(spec, self.device)
        bodies = list(spec.get("bodies", []))
        out = C.c_int64()
        _check(self.lib.lbm_batch_solve_bytes(C.byref(d), body_array(bodies), len(bodies),
                                              self._steps(spec, steps), C.byref(out)))
        return int(out.value)

    def admit(self, spec: dict, steps: int | None = None):
        """slot index, or None when the solve does not fit (budget or slots)"""
        d, _, _ = domain_desc(spec, self.device)
        bodies = list(spec.get("bodies", []))
        slot = C.c_int(-1)
        rc = self.lib.lbm_batch_admit(self.h, C.byref(d), body_array(bodies), len(bodies),
                                      self._steps(spec, steps), C.byref(slot))
        if rc == 2:  # LBM_ERR_OOM
            return None
        _check(rc)
        self.specs[slot.value] = spec
        return int(slot.value)

    def run(self, n: int = 1):
        _check(self.lib.lbm_batch_run(self.h, int(n)))

    def poll(self) -> list:
        cap = max(len(self.specs), 1)
        out = (C.c_int * cap)()
        cnt = C.c_int()
        _check(self.lib.lbm_batch_poll(self.h, out, cap, C.byref(cnt)))
        return [int(out[k]) for k in range(cnt.value)]

    def time(self, slot: int) -> int:
        return int(self.lib.lbm_batch_time(self.h, int(slot)))

    def force_torque(self, slot: int, kind: str = "static", first: int = 0, count: int | None = None):
        nb = len(self.specs[slot].get("bodies", []))
        if count is None:
            count = self.time(slot) - first
        out = np.zeros((count, max(nb, 1), 6))
        if nb and count:
            _check(self.lib.lbm_batch_get_force_torque(self.h, int(slot), int(first), int(count),
                                                       FT_KIND[kind], out.ctypes.data))
        return out[:, :nb]

    def release(self, slot: int):
        _check(self.lib.lbm_batch_release(self.h, int(slot)))
        self.specs.pop(slot, None)

    def usage(self):
        r = C.c_int()
        b = C.c_int64()
        _check(self.lib.lbm_batch_usage(self.h, C.byref(r), C.byref(b)))
        return int(r.value), int(b.value)
