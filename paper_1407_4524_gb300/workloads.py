"""Seeded synthetic problem descriptions shaped like the paper's test cases.

This module holds no arithmetic of the method: it only builds plain dicts
(lattice, sizes, relaxation time, edges, bodies) and seeded random body
placements / request traces.  Both the CUDA binding and the FP64 oracle take
these dicts, so they are the one thing the two sides share.

Problem-description keys (all sizes in lattice units, velocities in lattice
units per step):
  lattice    "D2Q9" | "D3Q19"
  n          (nx, ny) or (nx, ny, nz)
  tau        BGK relaxation time (Eq. LBE)
  rho0       reference density of the quasi-incompressible model (Sec. 2)
  eq         "incomp" (He-Luo, the paper's choice) | "standard"
  edges      {"x": "periodic" | (lo, hi), "y": ..., "z": ...}; kinds "wall",
             "inlet" (x-lo only), "outlet" (x-hi only)
  inlet      {"profile": "uniform" | "parabolic", "u": velocity (max if parabolic)}
  force      body-force density (gx, gy[, gz]) or absent
  u0         initial uniform velocity
  refill     "uB" (f^eq(rho_bar, u_B)) | "ubar" (f^eq(rho_bar, u_bar)) | "extrap"
             (quadratic extrapolation along the lattice direction nearest the normal)
  edge_rule  "link" (walls / inlet as half-way links) | "zouhe" (Zou-He nodes on the faces)
  bodies     list of {"shape": "cylinder" | "sphere" | "ellipse", "R", "X0", "U",
             "W", "halfway", "t0"; free bodies: "free", "density_ratio";
             ellipses: "R2" (second semi-axis), "theta0"}
  gravity    acceleration of the free bodies (lattice units)
  free_scheme "explicit" | "aidun" | "predictor": covered / uncovered sets of
             free bodies (Sec. 3, after Eq. ForceInMovement)
  precision  "fp64" | "fp32" | "fp16"  (CUDA side only)
"""
from __future__ import annotations

import math

import numpy as np


def channel_cylinder_2d(precision: str = "fp64") -> dict:
    """D2Q9 channel 200x80, tau 0.8, parabolic inflow u_max 0.05, zero-gradient
    outflow, no-slip walls, static cylinder R=8 at (40,40); 5000 steps."""
    return dict(
        name="channel_cylinder_2d", lattice="D2Q9", n=(200, 80), tau=0.8,
        edges={"x": ("inlet", "outlet"), "y": ("wall", "wall")},
        inlet={"profile": "parabolic", "u": 0.05},
        bodies=[dict(shape="cylinder", R=8.0, X0=(40.0, 40.0))],
        precision=precision, steps=5000,
    )


def poiseuille_2d(precision: str = "fp64", ny: int = 64, g: float = 1e-6, tau: float = 0.8) -> dict:
    """Periodic 1 x ny channel between halfway walls driven by a body force."""
    return dict(
        name="poiseuille_2d", lattice="D2Q9", n=(1, ny), tau=tau,
        edges={"x": "periodic", "y": ("wall", "wall")}, force=(g, 0.0),
        precision=precision, steps=int(6 * ny * ny / ((tau - 0.5) / 3.0)),
    )


def moving_cylinders_2d(precision: str = "fp32") -> dict:
    """D2Q9 periodic 512x256, tau 0.6, fluid at rest; cylinder R=12 translating
    at (0.02, 0) and cylinder R=10 rotating at 0.002; 20000 steps."""
    return dict(
        name="moving_cylinders_2d", lattice="D2Q9", n=(512, 256), tau=0.6,
        bodies=[dict(shape="cylinder", R=12.0, X0=(128.0, 64.0), U=(0.02, 0.0)),
                dict(shape="cylinder", R=10.0, X0=(384.0, 192.0), W=0.002)],
        precision=precision, steps=20000,
    )


def sphere_channel_3d(precision: str = "fp32") -> dict:
    """D3Q19 channel 256x128x128, tau 0.55, uniform inflow 0.04, zero-gradient
    outflow, periodic cross-section, static sphere R=12 at (64,64,64); the
    fluid starts as the uniform inflow stream (impulsive start)."""
    return dict(
        name="sphere_channel_3d", lattice="D3Q19", n=(256, 128, 128), tau=0.55,
        edges={"x": ("inlet", "outlet"), "y": "periodic", "z": "periodic"},
        inlet={"profile": "uniform", "u": 0.04}, u0=(0.04, 0.0, 0.0),
        bodies=[dict(shape="sphere", R=12.0, X0=(64.0, 64.0, 64.0))],
        precision=precision, steps=10000,
    )


def _wall_spacing(nx: int, width: float, edge_rule: str) -> float:
    """Lattice spacing of a channel of `width` across nx nodes: Zou-He walls
    sit on the outer node rows (nx - 1 spacings), half-way link walls half a
    spacing outside them (nx spacings)."""
    return width / (nx - 1) if edge_rule == "zouhe" else width / nx


def sedimenting_disc_2d(precision: str = "fp64", density_ratio: float = 1.01, steps: int = 20000,
                        edge_rule: str = "zouhe") -> dict:
    """The paper's sedimenting disc in lattice units: D2Q9 135 x 1073, tau 0.6,
    no-slip walls on every face (Zou-He nodes, the paper's edge treatment, or
    half-way links), a free disc of diameter d = W/4 falling under gravity.
    Physical data: W = 4 mm (135 nodes), H = 8 W, d = 1 mm, water (rho 1000,
    nu 1e-6 m^2/s), g = 9.81 m/s^2; nu_lattice = (tau - 1/2)/3 fixes the time
    step dt = nu_lattice dx^2 / nu, so g_lattice = g dt^2 / dx.  The centre
    starts 25 mm above the bottom and 0.76 mm off the channel axis."""
    nx, ny, tau = 135, 1073, 0.6
    dx = _wall_spacing(nx, 4e-3, edge_rule)
    nu_l = (tau - 0.5) / 3.0
    dt = nu_l * dx * dx / 1e-6
    g_l = 9.81 * dt * dt / dx
    R = 0.5e-3 / dx
    x0 = 0.5 * (nx - 1) + 7.6e-4 / dx
    y0 = 25e-3 / dx
    return dict(
        name="sedimenting_disc_2d", lattice="D2Q9", n=(nx, ny), tau=tau, edge_rule=edge_rule,
        edges={"x": ("wall", "wall"), "y": ("wall", "wall")}, gravity=(0.0, -g_l),
        bodies=[dict(shape="cylinder", R=R, X0=(x0, y0), free=True, density_ratio=float(density_ratio))],
        precision=precision, steps=steps,
    )


def sedimenting_ellipse_2d(precision: str = "fp64", density_ratio: float = 1.10, steps: int = 20000,
                           edge_rule: str = "zouhe") -> dict:
    """The paper's sedimenting ellipse in lattice units: D2Q9 135 x 1676, tau
    0.6, no-slip walls on every face (Zou-He nodes or half-way links), a free
    ellipse with major axis a = 1 mm (the full
    axis; semi-axes a/2 and a/4: aspect ratio 2), channel W = 4 a (blockage 4),
    H = 50 a, released at the channel axis 48 mm above the bottom at
    theta0 = pi/4, r_rho = 1.10; water and g as for the disc."""
    nx, ny, tau = 135, 1676, 0.6
    dx = _wall_spacing(nx, 4e-3, edge_rule)
    nu_l = (tau - 0.5) / 3.0
    dt = nu_l * dx * dx / 1e-6
    g_l = 9.81 * dt * dt / dx
    return dict(
        name="sedimenting_ellipse_2d", lattice="D2Q9", n=(nx, ny), tau=tau, edge_rule=edge_rule,
        edges={"x": ("wall", "wall"), "y": ("wall", "wall")}, gravity=(0.0, -g_l),
        bodies=[dict(shape="ellipse", R=0.5e-3 / dx, R2=0.25e-3 / dx, theta0=math.pi / 4,
                     X0=(0.5 * (nx - 1), 48e-3 / dx), free=True, density_ratio=float(density_ratio))],
        precision=precision, steps=steps,
    )


def _unit_vector(rng) -> np.ndarray:
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def _min_gap(p1, v1, r1, p2, v2, r2, L, steps) -> float:
    """smallest surface gap of two linear trajectories over [0, steps]
    (minimum image), sampled finely enough for |v| <= 0.02"""
    ts = np.linspace(0.0, steps, 201)
    d = (p1 - p2)[None, :] + ts[:, None] * (v1 - v2)[None, :]
    d -= L * np.floor(d / L + 0.5)
    return float(np.sqrt((d * d).sum(1)).min() - r1 - r2)


def sphere_swarm_3d(precision: str = "fp32", n=(512, 256, 256), n_bodies: int = 64,
                    seed: int = 1407, steps: int = 2000, r_range=(6.0, 12.0),
                    u_max: float = 0.02, w_max: float = 0.001) -> dict:
    """D3Q19 periodic box 512x256x256, tau 0.6, fluid at rest, 64 spheres of
    radius U[6,12]; even index static, odd index translating (|U| <= 0.02, uniform
    direction) and rotating (|W| <= 0.001); centres uniform, rejected if two
    trajectories come closer than R1 + R2 + 2 (+0.25 sampling margin) within
    ``steps`` steps."""
    rng = np.random.default_rng(seed)
    L = np.array(n, dtype=float)
    bodies = []
    tries = 0
    while len(bodies) < n_bodies:
        tries += 1
        if tries > 200000:
            raise RuntimeError("could not place spheres")
        k = len(bodies)
        R = float(rng.uniform(*r_range))
        X = rng.uniform(0.0, 1.0, 3) * L
        if k % 2 == 1:
            U = _unit_vector(rng) * rng.uniform(0.0, u_max)
            W = _unit_vector(rng) * rng.uniform(0.0, w_max)
        else:
            U = np.zeros(3)
            W = np.zeros(3)
        ok = True
        for b in bodies:
            if _min_gap(X, U, R, np.array(b["X0"]), np.array(b["U"]), b["R"], L, steps) < 2.25:
                ok = False
                break
        if ok:
            bodies.append(dict(shape="sphere", R=R, X0=tuple(map(float, X)),
                               U=tuple(map(float, U)), W=tuple(map(float, W))))
    return dict(name="sphere_swarm_3d", lattice="D3Q19", n=tuple(n), tau=0.6,
                bodies=bodies, precision=precision, steps=steps, seed=seed)


SERVING_D2Q9_SIZES = ((128, 64), (256, 128), (512, 256), (1024, 512))
SERVING_D3Q19_SIZES = ((64, 64, 64), (128, 64, 64), (192, 96, 96))


def serving_request(rng, lattice: str | None = None, precision: str = "fp16") -> dict:
    """One served solve: D2Q9 (channel, parabolic inflow, walls; fluid at
    rest) or D3Q19 (channel, uniform inflow, periodic cross-section; fluid
    starting as the inflow stream), one body of radius U[5,15] near x = nx/4,
    tau U[0.52,1.0], inflow U[0.01,0.05], steps U{2000..20000}."""
    if lattice is None:
        lattice = "D2Q9" if rng.uniform() < 0.5 else "D3Q19"
    tau = float(rng.uniform(0.52, 1.0))
    u_in = float(rng.uniform(0.01, 0.05))
    R = float(rng.uniform(5.0, 15.0))
    steps = int(rng.integers(2000, 20001))
    if lattice == "D2Q9":
        n = SERVING_D2Q9_SIZES[int(rng.integers(len(SERVING_D2Q9_SIZES)))]
        lo = max(n[0] / 4 - n[0] / 16, R + 3.0)
        xc = float(rng.uniform(lo, max(lo, n[0] / 4 + n[0] / 16)))
        yc = float(rng.uniform(R + 3.0, n[1] - 1 - R - 3.0))
        return dict(name="serving_2d", lattice=lattice, n=n, tau=tau,
                    edges={"x": ("inlet", "outlet"), "y": ("wall", "wall")},
                    inlet={"profile": "parabolic", "u": u_in},
                    bodies=[dict(shape="cylinder", R=R, X0=(xc, yc))],
                    precision=precision, steps=steps)
    n = SERVING_D3Q19_SIZES[int(rng.integers(len(SERVING_D3Q19_SIZES)))]
    lo = max(n[0] / 4 - n[0] / 16, R + 3.0)
    xc = float(rng.uniform(lo, max(lo, n[0] / 4 + n[0] / 16)))
    yc = float(rng.uniform(0.0, n[1]))
    zc = float(rng.uniform(0.0, n[2]))
    return dict(name="serving_3d", lattice=lattice, n=n, tau=tau,
                edges={"x": ("inlet", "outlet"), "y": "periodic", "z": "periodic"},
                inlet={"profile": "uniform", "u": u_in}, u0=(u_in, 0.0, 0.0),
                bodies=[dict(shape="sphere", R=R, X0=(xc, yc, zc))],
                precision=precision, steps=steps)


def serving_trace(seed: int = 4524, n_requests: int = 200, rate_hz: float = 20.0,
                  precision: str = "fp16") -> list:
    """Poisson arrivals (mean ``rate_hz``) of ``n_requests`` served solves."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n_requests):
        t += float(rng.exponential(1.0 / rate_hz))
        req = serving_request(rng, precision=precision)
        req["arrival_s"] = t
        req["id"] = k
        out.append(req)
    return out


def cells(spec: dict) -> int:
    n = tuple(spec["n"]) + (1,) * (3 - len(spec["n"]))
    return int(math.prod(n))


def with_precision(spec: dict, precision: str) -> dict:
    out = dict(spec)
    out["precision"] = precision
    return out
