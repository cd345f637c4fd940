"""ctypes wrapper of the FP64 oracle (test infrastructure; see package doc)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

# series row layout of or_get_series (per body per step)
SERIES_FIELDS = ("Fs", "Ts", "Fi", "Ti", "Fm", "Tm")

_EDGE = {"periodic": 0, "wall": 1, "inlet": 2, "outlet": 3}
_SHAPE = {"cylinder": 0, "sphere": 1, "ellipse": 2}


class _Desc(C.Structure):
    _fields_ = [
        ("q", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("eq", C.c_int), ("edge", C.c_int * 6), ("inlet_parabolic", C.c_int),
        ("has_force", C.c_int), ("refill", C.c_int),
        ("tau", C.c_double), ("rho0", C.c_double), ("u_in", C.c_double),
        ("g", C.c_double * 3), ("u0", C.c_double * 3), ("gravity", C.c_double * 3),
        ("edge_rule", C.c_int), ("free_scheme", C.c_int),
    ]


class _Body(C.Structure):
    _fields_ = [
        ("shape", C.c_int), ("halfway", C.c_int), ("invert", C.c_int), ("free", C.c_int),
        ("R", C.c_double), ("X0", C.c_double * 3), ("U", C.c_double * 3),
        ("W", C.c_double * 3), ("t0", C.c_longlong), ("density_ratio", C.c_double),
        ("R2", C.c_double), ("theta0", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c with gcc (FP contraction off) and return the path."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                           capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    P = C.c_void_p
    lib.or_create.restype = P
    lib.or_create.argtypes = [C.POINTER(_Desc)]
    lib.or_destroy.argtypes = [P]
    lib.or_set_bodies.argtypes = [P, C.POINTER(_Body), C.c_int]
    lib.or_set_f.argtypes = [P, P]
    lib.or_step.argtypes = [P, C.c_int]
    lib.or_time.restype = C.c_longlong
    lib.or_time.argtypes = [P]
    lib.or_fallbacks.restype = C.c_longlong
    lib.or_fallbacks.argtypes = [P]
    lib.or_extrapolated.restype = C.c_longlong
    lib.or_extrapolated.argtypes = [P]
    lib.or_mismatches.restype = C.c_longlong
    lib.or_mismatches.argtypes = [P]
    lib.or_get_series.argtypes = [P, C.c_longlong, C.c_longlong, P]
    for name in ("or_get_f", "or_get_fhat", "or_get_macro", "or_get_solid", "or_get_edge_me", "or_get_bodies"):
        getattr(lib, name).argtypes = [P, P]
    lib.or_links.restype = C.c_longlong
    lib.or_links.argtypes = [P, C.c_int, C.c_longlong, P, P, P]
    lib.or_lattice.argtypes = [C.c_int, P, P, P]
    lib.or_sincos.argtypes = [C.c_double, P, P]
    lib.or_threads.restype = C.c_int
    lib.or_threads.argtypes = []
    _lib = lib
    return lib


def threads() -> int:
    """threads the oracle's OpenMP loops use (1 if it was built without OpenMP)"""
    return int(_load().or_threads())


def sincos(x: float):
    """the oracle's own sin and cos (used for body orientations)"""
    lib = _load()
    s = C.c_double()
    c = C.c_double()
    lib.or_sincos(float(x), C.byref(s), C.byref(c))
    return s.value, c.value


def lattice_tables(q: int):
    """(c[Q,3] int, w[Q] float64, opp[Q] int) exactly as the oracle uses them."""
    lib = _load()
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q, dtype=np.float64)
    opp = np.zeros(q, dtype=np.int32)
    if lib.or_lattice(q, c.ctypes.data, w.ctypes.data, opp.ctypes.data) != 0:
        raise ValueError(f"unknown lattice Q={q}")
    return c, w, opp


def _edge_codes(spec):
    edges = spec.get("edges", {})
    out = []
    for ax in "xyz":
        e = edges.get(ax, "periodic")
        lo, hi = (e, e) if isinstance(e, str) else e
        out += [_EDGE[lo], _EDGE[hi]]
    return out


def _body_struct(b) -> _Body:
    s = _Body()
    s.shape = _SHAPE[b.get("shape", "sphere")]
    s.halfway = int(bool(b.get("halfway", False)))
    s.invert = int(bool(b.get("invert", False)))
    s.R = float(b["R"])
    for k in range(3):
        s.X0[k] = float(tuple(b["X0"])[k]) if k < len(b["X0"]) else 0.0
        s.U[k] = float(tuple(b.get("U", (0, 0, 0)))[k]) if k < len(b.get("U", (0, 0, 0))) else 0.0
    W = b.get("W", (0.0, 0.0, 0.0))
    if np.isscalar(W):
        W = (0.0, 0.0, float(W))
    for k in range(3):
        s.W[k] = float(W[k])
    s.t0 = int(b.get("t0", 0))
    s.free = int(bool(b.get("free", False)))
    s.density_ratio = float(b.get("density_ratio", 1.0))
    s.R2 = float(b.get("R2", b["R"]))
    s.theta0 = float(b.get("theta0", 0.0))
    return s


class Oracle:
    """One FP64 oracle domain built from a problem description dict.

    Required keys: ``lattice`` ("D2Q9"/"D3Q19"), ``n`` (nx, ny[, nz]), ``tau``.
    Optional: ``rho0``, ``eq`` ("incomp"/"standard"), ``edges`` (per axis
    "periodic" | (lo, hi) kinds among "wall", "inlet", "outlet"), ``inlet``
    ({"profile": "uniform"/"parabolic", "u": ...}), ``force``, ``u0``,
    ``refill`` ("uB"/"ubar"/"extrap"), ``gravity`` (acceleration of free bodies),
    ``free_scheme`` ("explicit" | "aidun" | "predictor": how free bodies take
    the covered / uncovered sets of their force, Sec. 3),
    ``edge_rule`` ("link": wall / inlet faces as half-way links; "zouhe": Zou-He
    nodes on the faces),
    ``bodies`` (list of dicts: shape, R, X0, U, W, halfway, invert, t0, free,
    density_ratio; ellipses: shape "ellipse", R and R2 the semi-axes, theta0).
    """

    def __init__(self, spec: dict):
        lib = _load()
        self.lib = lib
        q = {"D2Q9": 9, "D3Q19": 19}[spec["lattice"]]
        n = tuple(spec["n"]) + (1,) * (3 - len(spec["n"]))
        d = _Desc()
        d.q, d.nx, d.ny, d.nz = q, n[0], n[1], n[2]
        d.eq = {"incomp": 0, "standard": 1}[spec.get("eq", "incomp")]
        for k, v in enumerate(_edge_codes(spec)):
            d.edge[k] = v
        inlet = spec.get("inlet", {})
        d.inlet_parabolic = int(inlet.get("profile", "uniform") == "parabolic")
        d.u_in = float(inlet.get("u", 0.0))
        g = spec.get("force")
        d.has_force = int(g is not None)
        for k in range(3):
            d.g[k] = float(g[k]) if g is not None and k < len(g) else 0.0
        u0 = tuple(spec.get("u0", (0.0, 0.0, 0.0)))
        for k in range(3):
            d.u0[k] = float(u0[k]) if k < len(u0) else 0.0
        d.refill = {"uB": 0, "ubar": 1, "extrap": 2}[spec.get("refill", "uB")]
        d.edge_rule = {"link": 0, "zouhe": 1}[spec.get("edge_rule", "link")]
        d.free_scheme = {"explicit": 0, "aidun": 1, "predictor": 2}[spec.get("free_scheme", "explicit")]
        gv = tuple(spec.get("gravity", (0.0, 0.0, 0.0)))
        for k in range(3):
            d.gravity[k] = float(gv[k]) if k < len(gv) else 0.0
        d.tau = float(spec["tau"])
        d.rho0 = float(spec.get("rho0", 1.0))
        h = lib.or_create(C.byref(d))
        if not h:
            raise ValueError("oracle rejected the problem description")
        self.h = C.c_void_p(h)
        self.q, self.shape = q, n
        self.N = n[0] * n[1] * n[2]
        self.bodies = list(spec.get("bodies", []))
        if self.bodies:
            arr = (_Body * len(self.bodies))(*[_body_struct(b) for b in self.bodies])
            rc = lib.or_set_bodies(self.h, arr, len(self.bodies))
            if rc:
                raise ValueError(f"or_set_bodies failed ({rc})")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.or_destroy(h)
            self.h = None

    # -- stepping -------------------------------------------------------------
    def step(self, n: int = 1):
        rc = self.lib.or_step(self.h, int(n))
        if rc:
            raise RuntimeError(f"or_step failed ({rc})")

    @property
    def t(self) -> int:
        return int(self.lib.or_time(self.h))

    @property
    def fallbacks(self) -> int:
        return int(self.lib.or_fallbacks(self.h))

    def mismatches(self) -> int:
        """free_scheme "predictor": nodes whose covering or uncovering the
        predicted displacement got wrong so far"""
        return int(self.lib.or_mismatches(self.h))

    def extrapolated(self) -> int:
        """Uncovered nodes refilled by extrapolation so far (refill "extrap")."""
        return int(self.lib.or_extrapolated(self.h))

    # -- state ----------------------------------------------------------------
    def _grid(self, arr, lead):
        nx, ny, nz = self.shape
        return arr.reshape(lead + (nz, ny, nx))

    def f(self) -> np.ndarray:
        """pre-collision populations f(t), shape [Q, nz, ny, nx]"""
        out = np.empty(self.q * self.N)
        self.lib.or_get_f(self.h, out.ctypes.data)
        return self._grid(out, (self.q,))

    def fhat(self) -> np.ndarray:
        """post-collision populations fhat(t) (0 at solid nodes)"""
        out = np.empty(self.q * self.N)
        self.lib.or_get_fhat(self.h, out.ctypes.data)
        return self._grid(out, (self.q,))

    def set_f(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        assert f.size == self.q * self.N
        self.lib.or_set_f(self.h, f.ctypes.data)

    def macro(self) -> np.ndarray:
        """rho, ux, uy, uz of f(t), shape [4, nz, ny, nx] (0 at solid nodes)"""
        out = np.empty(4 * self.N)
        self.lib.or_get_macro(self.h, out.ctypes.data)
        return self._grid(out, (4,))

    def solid(self) -> np.ndarray:
        """owning body index of every node at time t, -1 for fluid"""
        out = np.empty(self.N, dtype=np.int32)
        self.lib.or_get_solid(self.h, out.ctypes.data)
        return self._grid(out, ())

    def body_state(self) -> np.ndarray:
        """[n_bodies, 9]: X(t), U(t), W(t)"""
        nb = len(self.bodies)
        out = np.zeros(max(nb, 1) * 9)
        self.lib.or_get_bodies(self.h, out.ctypes.data)
        return out.reshape(-1, 9)[:nb]

    def edge_me(self) -> np.ndarray:
        out = np.empty(6)
        self.lib.or_get_edge_me(self.h, out.ctypes.data)
        return out

    def series(self, first: int = 0, count: int | None = None) -> np.ndarray:
        """[count, n_bodies, 18]: Fs, Ts, Fi, Ti, Fm, Tm (3 components each)"""
        nb = len(self.bodies)
        if count is None:
            count = self.t - first
        out = np.zeros((count, max(nb, 1), 18))
        if nb and count:
            rc = self.lib.or_get_series(self.h, first, count, out.ctypes.data)
            if rc:
                raise ValueError("series range out of bounds")
        return out[:, :nb]

    def force_torque(self, kind: str = "static") -> np.ndarray:
        """[steps, n_bodies, 6] (F, T) in one of the paper's forms:
        static (Eqs. flow_force_2/flow_torque_2), lattice (Eqs. ForceInMovement/
        TorqueInMovement), moving (Eqs. ForceInMovementMovingFrame/...)."""
        s = self.series()
        if kind == "static":
            return s[..., 0:6].copy()
        if kind == "impulsive":
            return s[..., 6:12].copy()
        if kind == "lattice":
            return s[..., 0:6] + s[..., 6:12]
        if kind == "moving":
            return s[..., 12:18].copy()
        raise ValueError(kind)

    def links(self, body: int):
        """(cells, dirs, deltas) of the body's cut links at time t"""
        cnt = int(self.lib.or_links(self.h, body, 0, None, None, None))
        cells = np.zeros(cnt, dtype=np.int64)
        dirs = np.zeros(cnt, dtype=np.int32)
        deltas = np.zeros(cnt)
        self.lib.or_links(self.h, body, cnt, cells.ctypes.data, dirs.ctypes.data, deltas.ctypes.data)
        return cells, dirs, deltas
