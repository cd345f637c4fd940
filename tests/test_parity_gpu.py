"""GPU path vs FP64 oracle, element by element on the same seeded inputs.

Cases span several CUDA blocks and ragged tails (sizes not multiples of the
block width), both lattices, every edge kind, static / translating /
rotating bodies (including bodies that straddle a periodic seam), both
equilibria, all three refill rules and all three precision modes.  FP64 mode must
reproduce the oracle to the benchmark spec's tolerance (it is built to be
bit-identical); FP32 / FP16 modes to the stated reduced-precision tolerance.
"""
import numpy as np
import pytest

from parity_util import (TOL_FP16_FT, TOL_FP16_POP, TOL_FP64_FT, TOL_FP64_POP, TOL_RED_FT, TOL_RED_POP,
                         ft_rel_error, pop_error, report)

pytestmark = pytest.mark.gpu


def _run_both(oracle_mod, spec, steps):
    from paper_1407_4524_gb300 import lbm
    dom = lbm.Domain(spec, device=0)
    dom.step(steps)
    ref = oracle_mod.Oracle(spec)
    ref.step(steps)
    return dom, ref


def _compare(dom, ref, pop_tol, ft_tol, kinds=("static", "lattice", "moving"), spec=None):
    solid = ref.solid()
    assert np.array_equal(dom.solid(), solid)
    perr = pop_error(dom.populations(), ref.fhat(), solid)
    assert perr <= pop_tol, f"populations differ by {perr:.3e}"
    out = {"pop": perr}
    if ref.bodies:
        for kind in kinds:
            e = ft_rel_error(dom.force_torque(kind), ref.force_torque(kind), spec=spec or dom.spec)
            assert e <= ft_tol, f"{kind} force/torque rel error {e:.3e}"
            out[kind] = e
    return out


CASES_2D = {
    "channel_cylinder": dict(
        lattice="D2Q9", n=(61, 29), tau=0.8, edges={"x": ("inlet", "outlet"), "y": ("wall", "wall")},
        inlet={"profile": "parabolic", "u": 0.05}, bodies=[dict(shape="cylinder", R=6.3, X0=(15.4, 14.2))]),
    "channel_cylinder_even": dict(  # even nx: FP16 node pairs at the inlet, outlet and walls
        lattice="D2Q9", n=(62, 30), tau=0.7, edges={"x": ("inlet", "outlet"), "y": ("wall", "wall")},
        inlet={"profile": "parabolic", "u": 0.05}, u0=(0.02, 0.0),
        bodies=[dict(shape="cylinder", R=5.7, X0=(17.2, 14.6))]),
    "channel_cylinder_64": dict(  # 16-byte rows: stream-collide from staged rows (FP32 and FP16)
        lattice="D2Q9", n=(64, 30), tau=0.7, edges={"x": ("inlet", "outlet"), "y": ("wall", "wall")},
        inlet={"profile": "parabolic", "u": 0.05}, u0=(0.02, 0.0),
        bodies=[dict(shape="cylinder", R=5.7, X0=(17.2, 14.6))]),
    "long_rows_periodic": dict(  # rows of several staging segments, the last one partial
        lattice="D2Q9", n=(328, 24), tau=0.65, u0=(0.03, -0.01),
        bodies=[dict(shape="cylinder", R=4.5, X0=(300.3, 11.2), U=(0.03, 0.0))]),
    "ellipse_channel": dict(  # static ellipse at 45 degrees: Delta in the rotated, scaled axes
        lattice="D2Q9", n=(64, 34), tau=0.7, edges={"x": ("inlet", "outlet"), "y": ("wall", "wall")},
        inlet={"profile": "parabolic", "u": 0.05},
        bodies=[dict(shape="ellipse", R=9.3, R2=4.4, theta0=0.785398, X0=(20.6, 16.8))]),
    "ellipse_rotating": dict(  # rotation alone covers and uncovers nodes
        lattice="D2Q9", n=(48, 46), tau=0.65, u0=(0.02, 0.0),
        bodies=[dict(shape="ellipse", R=9.1, R2=3.7, theta0=0.3, X0=(23.2, 22.6), W=0.006, U=(0.01, 0.0))]),
    "moving_cylinders_periodic": dict(
        lattice="D2Q9", n=(97, 66), tau=0.6,
        bodies=[dict(shape="cylinder", R=8.2, X0=(6.3, 20.4), U=(0.06, -0.03)),  # crosses the seam
                dict(shape="cylinder", R=7.0, X0=(60.0, 45.0), W=0.004)]),
    "standard_eq_walls": dict(
        lattice="D2Q9", n=(48, 40), tau=0.7, eq="standard", u0=(0.03, 0.0),
        edges={"x": "periodic", "y": ("wall", "wall")},
        bodies=[dict(shape="cylinder", R=5.1, X0=(20.5, 19.3), U=(0.04, 0.0), W=-0.003)]),
    "refill_ubar": dict(
        lattice="D2Q9", n=(45, 41), tau=0.9, refill="ubar", u0=(0.01, 0.02),
        bodies=[dict(shape="cylinder", R=6.6, X0=(22.2, 20.1), U=(0.07, 0.05))]),
    "refill_extrap": dict(  # extrapolation refill; the static neighbour forces some fallbacks
        lattice="D2Q9", n=(52, 38), tau=0.8, refill="extrap", u0=(0.01, -0.02),
        edges={"x": "periodic", "y": ("wall", "wall")},
        bodies=[dict(shape="cylinder", R=6.0, X0=(14.0, 19.0)),
                dict(shape="cylinder", R=6.0, X0=(28.3, 19.4), U=(0.03, 0.0), W=0.004)]),
    "refill_extrap_ellipse": dict(  # normal from the rotated ellipse's gradient at t+1
        lattice="D2Q9", n=(50, 44), tau=0.7, refill="extrap", u0=(0.02, 0.0),
        bodies=[dict(shape="ellipse", R=8.7, R2=4.1, theta0=0.9, X0=(24.1, 21.7), W=0.008, U=(0.03, 0.02))]),
    "zouhe_poiseuille": dict(  # Zou-He walls on the node rows 0 and ny - 1, body force
        lattice="D2Q9", n=(5, 33), tau=0.8, force=(1e-5, 0.0), edge_rule="zouhe",
        edges={"x": "periodic", "y": ("wall", "wall")}),
    "zouhe_channel_cylinder": dict(  # Zou-He parabolic inlet and walls, zero-gradient outlet
        lattice="D2Q9", n=(61, 29), tau=0.7, edge_rule="zouhe", u0=(0.02, 0.0),
        edges={"x": ("inlet", "outlet"), "y": ("wall", "wall")}, inlet={"profile": "parabolic", "u": 0.05},
        bodies=[dict(shape="cylinder", R=6.3, X0=(15.4, 14.2))]),
    "zouhe_box_rotating": dict(  # closed Zou-He box: every corner; a rotating ellipse
        lattice="D2Q9", n=(41, 37), tau=0.75, edge_rule="zouhe", eq="standard",
        edges={"x": ("wall", "wall"), "y": ("wall", "wall")},
        bodies=[dict(shape="ellipse", R=9.0, R2=5.2, theta0=0.4, X0=(20.3, 18.2), W=0.01)]),
    "halfway_body": dict(
        lattice="D2Q9", n=(40, 33), tau=0.66, u0=(0.03, 0.01),
        bodies=[dict(shape="cylinder", R=5.5, X0=(19.0, 16.5), halfway=True)]),
    "poiseuille_1col": dict(
        lattice="D2Q9", n=(1, 64), tau=0.8, edges={"x": "periodic", "y": ("wall", "wall")}, force=(1e-6, 0.0)),
    "no_bodies_ragged": dict(lattice="D2Q9", n=(37, 23), tau=0.55, u0=(0.02, -0.01)),
    "node_on_surface": dict(  # integer centre and radius: nodes exactly on the surface, Delta = 1 links
        lattice="D2Q9", n=(40, 40), tau=0.7, u0=(0.04, 0.01),
        bodies=[dict(shape="cylinder", R=5.0, X0=(20.0, 20.0))]),
    "two_bodies_close": dict(  # 2-cell surface gap: fluid nodes with links to both bodies
        lattice="D2Q9", n=(48, 36), tau=0.75, u0=(0.03, 0.0),
        bodies=[dict(shape="cylinder", R=6.0, X0=(15.0, 18.0)),
                dict(shape="cylinder", R=6.0, X0=(29.2, 18.4), U=(0.0, 0.03))]),
}

CASES_3D = {
    "channel_sphere": dict(
        lattice="D3Q19", n=(42, 26, 22), tau=0.55, edges={"x": ("inlet", "outlet")},
        inlet={"u": 0.04}, bodies=[dict(shape="sphere", R=5.3, X0=(12.4, 13.1, 10.6))]),
    "moving_spheres_periodic": dict(
        lattice="D3Q19", n=(40, 34, 30), tau=0.6,
        bodies=[dict(shape="sphere", R=6.2, X0=(9.0, 10.0, 8.0)),
                dict(shape="sphere", R=4.7, X0=(30.0, 24.5, 2.2), U=(0.05, -0.02, 0.04), W=(0.002, 0.0, -0.003)),
                dict(shape="sphere", R=3.9, X0=(28.0, 7.0, 20.0), U=(-0.03, 0.04, 0.01))]),
    "single_cell_box": dict(lattice="D3Q19", n=(1, 1, 1), tau=0.8, u0=(0.01, 0.02, -0.03)),
    "refill_extrap_spheres": dict(
        lattice="D3Q19", n=(36, 30, 28), tau=0.7, refill="extrap", u0=(0.01, 0.0, 0.01),
        edges={"x": "periodic", "y": ("wall", "wall"), "z": "periodic"},
        bodies=[dict(shape="sphere", R=5.2, X0=(9.4, 15.2, 13.8), U=(0.06, 0.0, -0.04)),
                dict(shape="sphere", R=4.1, X0=(27.0, 8.0, 3.0), U=(-0.04, 0.0, 0.05), W=(0.0, 0.004, 0.0))]),
    "walled_channel_sphere": dict(  # 16-byte rows, walls on y, inlet / outlet on x
        lattice="D3Q19", n=(48, 20, 18), tau=0.62, edges={"x": ("inlet", "outlet"), "y": ("wall", "wall")},
        inlet={"u": 0.03}, u0=(0.03, 0.0, 0.0), bodies=[dict(shape="sphere", R=4.6, X0=(14.2, 9.7, 8.9))]),
    "ellipse_3d_rotating": dict(  # elliptic cylinder along z in D3Q19, rotating about z
        lattice="D3Q19", n=(36, 34, 8), tau=0.7, u0=(0.02, 0.01, 0.0),
        bodies=[dict(shape="ellipse", R=8.2, R2=4.6, theta0=1.1, X0=(17.4, 16.9, 0.0), W=(0.0, 0.0, 0.005))]),
    "zouhe_duct_sphere": dict(  # Zou-He inlet, walls on y and z (3-D edges), outlet
        lattice="D3Q19", n=(40, 21, 19), tau=0.65, edge_rule="zouhe", u0=(0.03, 0.0, 0.0),
        edges={"x": ("inlet", "outlet"), "y": ("wall", "wall"), "z": ("wall", "wall")}, inlet={"u": 0.03},
        bodies=[dict(shape="sphere", R=4.8, X0=(13.2, 10.4, 9.3))]),
    "zouhe_closed_box": dict(  # every 3-D edge and corner; a rotating sphere
        lattice="D3Q19", n=(23, 21, 20), tau=0.7, edge_rule="zouhe",
        edges={"x": ("wall", "wall"), "y": ("wall", "wall"), "z": ("wall", "wall")},
        bodies=[dict(shape="sphere", R=5.1, X0=(11.3, 10.2, 9.8), W=(0.004, -0.006, 0.008))]),
    "walled_box_cylinder3d": dict(
        lattice="D3Q19", n=(30, 28, 9), tau=0.7, u0=(0.02, 0.01, 0.0),
        edges={"x": ("wall", "wall"), "y": ("wall", "wall"), "z": "periodic"},
        bodies=[dict(shape="cylinder", R=6.0, X0=(14.3, 13.6, 0.0), W=(0.0, 0.0, 0.003))]),
}


@pytest.mark.parametrize("name", sorted(CASES_2D))
def test_fp64_parity_2d(oracle_mod, name):
    spec = dict(CASES_2D[name], precision="fp64")
    dom, ref = _run_both(oracle_mod, spec, 120)
    _compare(dom, ref, TOL_FP64_POP, TOL_FP64_FT)
    st = dom.stats()
    assert st["fallback_links"] == ref.fallbacks


@pytest.mark.parametrize("name", sorted(CASES_3D))
def test_fp64_parity_3d(oracle_mod, name):
    spec = dict(CASES_3D[name], precision="fp64")
    dom, ref = _run_both(oracle_mod, spec, 40)
    _compare(dom, ref, TOL_FP64_POP, TOL_FP64_FT)


def test_fp64_is_bit_identical(oracle_mod):
    """The FP64 mode evaluates every formula in the oracle's operation order."""
    spec = dict(CASES_3D["moving_spheres_periodic"], precision="fp64")
    dom, ref = _run_both(oracle_mod, spec, 25)
    solid = ref.solid()
    fl = solid < 0
    assert np.array_equal(dom.populations()[:, fl], ref.fhat()[:, fl])
    assert np.array_equal(dom.series(), ref.series())


# every case in both reduced-precision modes: odd and even nx (FP16 storage
# moves node pairs when nx is even), all edge kinds (walls on x and y, inlet,
# outlet), both equilibria, forcing, moving and static bodies
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("name", sorted(CASES_2D))
def test_reduced_precision_2d(oracle_mod, name, prec):
    spec = dict(CASES_2D[name], precision=prec)
    dom, ref = _run_both(oracle_mod, spec, 120)
    pop_tol = TOL_RED_POP if prec == "fp32" else TOL_FP16_POP
    ft_tol = TOL_RED_FT if prec == "fp32" else TOL_FP16_FT
    report(f"{name}_{prec}_120", _compare(dom, ref, 1e9, 1e9))
    _compare(dom, ref, pop_tol, ft_tol)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("name", sorted(CASES_3D))
def test_reduced_precision_3d(oracle_mod, name, prec):
    spec = dict(CASES_3D[name], precision=prec)
    dom, ref = _run_both(oracle_mod, spec, 40)
    pop_tol = TOL_RED_POP if prec == "fp32" else TOL_FP16_POP
    ft_tol = TOL_RED_FT if prec == "fp32" else TOL_FP16_FT
    report(f"{name}_{prec}_40", _compare(dom, ref, 1e9, 1e9))
    _compare(dom, ref, pop_tol, ft_tol)


def test_zero_steps_and_empty_reads(oracle_mod):
    from paper_1407_4524_gb300 import lbm
    spec = dict(CASES_2D["channel_cylinder"], precision="fp64")
    dom = lbm.Domain(spec, device=0)
    dom.step(0)
    assert dom.t == 0
    assert dom.force_torque("static").shape == (0, 1, 6)
    ref = oracle_mod.Oracle(spec)
    fl = ref.solid() < 0
    assert np.array_equal(dom.populations()[:, fl], ref.fhat()[:, fl])


def test_invalid_bodies_rejected():
    from paper_1407_4524_gb300 import lbm
    base = dict(lattice="D2Q9", n=(40, 30), tau=0.7, precision="fp32",
                edges={"x": ("inlet", "outlet"), "y": ("wall", "wall")})
    bad = [
        [dict(shape="cylinder", R=5.0, X0=(3.0, 15.0))],                      # touches the inlet face
        [dict(shape="cylinder", R=5.0, X0=(12.0, 15.0)),
         dict(shape="cylinder", R=5.0, X0=(22.5, 15.0))],                     # surface gap < 2
        [dict(shape="sphere", R=4.0, X0=(20.0, 15.0))],                       # sphere on D2Q9
        [dict(shape="cylinder", R=4.0, X0=(20.0, 15.0), U=(0.01, 0.0))],       # translating along a non-periodic axis
    ]
    for bodies in bad:
        with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
            lbm.Domain(dict(base, bodies=bodies), device=0)
    dom = lbm.Domain(dict(base, bodies=[dict(shape="cylinder", R=4.0, X0=(20.0, 15.0))]), device=0)
    dom.step(1)
    with pytest.raises(lbm.LbmError, match="LBM_ERR_STATE"):
        dom.set_bodies([dict(shape="cylinder", R=4.0, X0=(20.0, 15.0))])
    with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
        dom.force_torque("static", first=0, count=5)


# With LBM_STAGED=1, reduced-precision domains whose rows are 16-byte aligned
# stream-collide from rows staged in shared memory by bulk copies (the default
# kernels load straight from global memory).  Same arithmetic per node: the
# results must agree bit for bit.
def _staged_cases():
    out = []
    for dim, cases in (("2d", CASES_2D), ("3d", CASES_3D)):
        for name in sorted(cases):
            nx = cases[name]["n"][0]
            for prec, s in (("fp32", 4), ("fp16", 2)):
                if nx >= 32 and (nx * s) % 16 == 0:
                    out.append((dim, name, prec))
    return out


@pytest.mark.parametrize("dim,name,prec", _staged_cases())
def test_staged_rows_bitwise(monkeypatch, dim, name, prec):
    from paper_1407_4524_gb300 import lbm
    spec = dict((CASES_2D if dim == "2d" else CASES_3D)[name], precision=prec)
    out = {}
    for staged in ("1", "0"):
        monkeypatch.setenv("LBM_STAGED", staged)
        dom = lbm.Domain(spec, device=0)
        dom.step(60)
        out[staged] = (dom.populations(), dom.series() if dom.bodies else None, dom.solid(), dom.stats())
        dom.close()
    assert out["1"][3]["timeouts"] == 0
    fl = out["1"][2] < 0
    assert np.array_equal(out["1"][0][:, fl], out["0"][0][:, fl])
    if out["1"][1] is not None:
        assert np.array_equal(out["1"][1], out["0"][1])


def test_unstable_solve_is_reported():
    """A flow beyond the stability check (|u| > 0.3 at a boundary node) makes
    the force/torque read of that solve fail with LBM_ERR_UNSTABLE."""
    from paper_1407_4524_gb300 import lbm
    for prec in ("fp32", "fp16"):
        spec = dict(lattice="D2Q9", n=(64, 32), tau=0.51, u0=(0.35, 0.0), precision=prec,
                    bodies=[dict(shape="cylinder", R=5.0, X0=(32.3, 16.2))])
        dom = lbm.Domain(spec, device=0)
        dom.step(3)
        assert dom.stats()["unstable"] == 1
        with pytest.raises(lbm.LbmError, match="LBM_ERR_UNSTABLE"):
            dom.force_torque("static")
        dom.close()
    calm = dict(CASES_2D["channel_cylinder"], precision="fp32")
    dom = lbm.Domain(calm, device=0)
    dom.step(20)
    assert dom.stats()["unstable"] == 0
    dom.close()


def test_staged_wait_expiry_is_reported(monkeypatch):
    """The staged kernel's mbarrier waits are bounded (one second): with the
    test hook its stages never fill, every block gives up, and the solve's
    reads return LBM_ERR_TIMEOUT; the context stays usable."""
    from paper_1407_4524_gb300 import lbm
    spec = dict(CASES_2D["channel_cylinder_64"], precision="fp32")
    monkeypatch.setenv("LBM_STAGED", "1")
    monkeypatch.setenv("LBM_STAGED_TEST_EXPIRE", "1")
    dom = lbm.Domain(spec, device=0)
    dom.step(1)
    assert dom.stats()["timeouts"] == 1
    with pytest.raises(lbm.LbmError, match="LBM_ERR_TIMEOUT"):
        dom.force_torque("static")
    dom.close()
    monkeypatch.delenv("LBM_STAGED_TEST_EXPIRE")
    dom = lbm.Domain(spec, device=0)  # same process, same context: works
    dom.step(5)
    assert dom.stats()["timeouts"] == 0
    assert np.isfinite(dom.force_torque("static")).all()
    dom.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("dim,name", [("2d", "refill_extrap"), ("2d", "refill_extrap_ellipse"),
                                      ("3d", "refill_extrap_spheres")])
def test_extrapolation_refill_choices_match(oracle_mod, dim, name, prec):
    """The extrapolation refill takes the same decisions as the oracle in every
    precision (normal, direction and fallback are evaluated in FP64 from the
    pose): as many nodes extrapolated, as many uncovered."""
    spec = dict((CASES_2D if dim == "2d" else CASES_3D)[name], precision=prec)
    steps = 120 if dim == "2d" else 40
    dom, ref = _run_both(oracle_mod, spec, steps)
    st = dom.stats()
    assert st["extrapolated"] == ref.extrapolated() > 0
    if name == "refill_extrap":  # trailing side next to the static body: some fallbacks to the equilibrium rule
        assert st["uncovered"] > st["extrapolated"]
