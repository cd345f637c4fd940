"""The two-node stream-collide kernel (reduced precision, even nx, no body
force, periodic y and z) against the single-node kernel (LBM_PAIR=0): the same
populations, force/torque series and moments bit for bit, over fully periodic
boxes and x-face channels, both lattices, static / moving / free bodies, rows
that end inside a warp, and both edge rules; and against the FP64 oracle to the
reduced-precision tolerance."""
import os

import numpy as np
import pytest

from parity_util import TOL_FP16_FT, TOL_FP16_POP, TOL_RED_FT, TOL_RED_POP, ft_rel_error, pop_error

pytestmark = pytest.mark.gpu

CASES = {
    "box_moving_spheres": dict(  # 70: the last warp of a row is partial
        lattice="D3Q19", n=(70, 40, 36), tau=0.6, u0=(0.01, -0.005, 0.002),
        bodies=[dict(shape="sphere", R=6.2, X0=(20.4, 19.6, 17.3), U=(0.02, 0.0, -0.01), W=(0.0, 0.002, 0.0)),
                dict(shape="sphere", R=5.1, X0=(52.2, 12.7, 18.9)),
                dict(shape="sphere", R=4.4, X0=(60.3, 30.1, 9.5), U=(-0.015, 0.01, 0.0))]),
    "box_seam": dict(  # a sphere across the periodic x seam (lane 0's left element wraps)
        lattice="D3Q19", n=(128, 28, 26), tau=0.7,
        bodies=[dict(shape="sphere", R=5.3, X0=(1.2, 11.4, 10.7), U=(-0.02, 0.0, 0.0))]),
    "channel_link": dict(  # x faces: inlet / outlet rows fall back to the single-node code
        lattice="D3Q19", n=(96, 30, 28), tau=0.6, edges={"x": ("inlet", "outlet"), "y": "periodic", "z": "periodic"},
        inlet={"profile": "uniform", "u": 0.04}, u0=(0.04, 0.0, 0.0),
        bodies=[dict(shape="sphere", R=6.4, X0=(30.2, 14.6, 13.9))]),
    "channel_wide": dict(  # x faces: many interior warps
        lattice="D3Q19", n=(250, 26, 24), tau=0.6, edges={"x": ("inlet", "outlet"), "y": "periodic", "z": "periodic"},
        inlet={"profile": "uniform", "u": 0.04}, u0=(0.04, 0.0, 0.0),
        bodies=[dict(shape="sphere", R=6.4, X0=(100.2, 12.6, 11.9))]),
    "channel_zouhe": dict(
        lattice="D3Q19", n=(130, 28, 28), tau=0.65, edge_rule="zouhe",
        edges={"x": ("inlet", "wall"), "y": "periodic", "z": "periodic"},
        inlet={"profile": "uniform", "u": 0.03}, u0=(0.01, 0.0, 0.0),
        bodies=[dict(shape="sphere", R=5.6, X0=(40.3, 12.2, 11.5), U=(0.0, 0.01, 0.0))]),
    "d2q9_periodic": dict(
        lattice="D2Q9", n=(98, 50), tau=0.7, u0=(0.03, 0.01),
        bodies=[dict(shape="cylinder", R=7.2, X0=(30.6, 24.3), U=(0.02, -0.01), W=0.002),
                dict(shape="ellipse", R=8.1, R2=4.2, theta0=0.5, X0=(70.2, 20.4), W=-0.001)]),
    "d2q9_channel_walls": dict(  # walls on y: the face rows fall back (general face mode)
        lattice="D2Q9", n=(130, 42), tau=0.6, edges={"x": ("inlet", "outlet"), "y": ("wall", "wall")},
        inlet={"profile": "parabolic", "u": 0.05}, bodies=[dict(shape="cylinder", R=6.3, X0=(32.4, 20.2))]),
    "d3q19_box_walls": dict(  # walls on z, periodic x and y
        lattice="D3Q19", n=(72, 30, 28), tau=0.7, edges={"z": ("wall", "wall")}, u0=(0.02, 0.0, 0.0),
        bodies=[dict(shape="sphere", R=5.2, X0=(30.3, 14.1, 13.6), U=(0.01, 0.0, 0.0))]),
    "free_spheres": dict(
        lattice="D3Q19", n=(40, 34, 32), tau=0.8, u0=(0.0, 0.0, 0.0),
        bodies=[dict(shape="sphere", R=5.1, X0=(12.6, 14.2, 15.1), U=(0.01, 0.0, -0.005), free=True,
                     density_ratio=2.0),
                dict(shape="sphere", R=4.2, X0=(28.3, 22.7, 13.6), free=True, density_ratio=0.8)]),
}
STEPS = 40


# kernel variants: the single-node kernel, the two-node kernel
VARIANTS = {"single": {"LBM_PAIR": "0"}, "pair": {"LBM_PAIR": "1"}}


def _run(spec, variant):
    from paper_1407_4524_gb300 import lbm
    env = VARIANTS[variant]
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        dom = lbm.Domain(spec, device=0)
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v
    dom.step(STEPS)
    out = dict(f=dom.populations(), series=dom.series(), body=dom.body_state(), mac=dom.macros())
    dom.close()
    return out


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_pair_kernel_bit_identical(name, prec):
    spec = dict(CASES[name], precision=prec)
    a = _run(spec, "pair")
    b = _run(spec, "single")
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("name", ["box_moving_spheres", "channel_zouhe", "d2q9_periodic", "d2q9_channel_walls"])
def test_pair_kernel_vs_oracle(oracle_mod, name, prec):
    from paper_1407_4524_gb300 import lbm
    spec = dict(CASES[name], precision=prec)
    dom = lbm.Domain(spec, device=0)
    dom.step(STEPS)
    ref = oracle_mod.Oracle(spec)
    ref.step(STEPS)
    solid = ref.solid()
    perr = pop_error(dom.populations(), ref.fhat(), solid)
    assert perr <= (TOL_RED_POP if prec == "fp32" else TOL_FP16_POP), perr
    for kind in ("static", "lattice", "moving"):
        e = ft_rel_error(dom.force_torque(kind), ref.force_torque(kind), spec=spec)
        assert e <= (TOL_RED_FT if prec == "fp32" else TOL_FP16_FT), (kind, e)
