"""GPU vs FP64 oracle at the benchmark configurations' full sizes.

* channel + cylinder, D2Q9 200x80, FP64, all 5000 steps: bit-identical
  populations and force/torque series;
* moving cylinders, D2Q9 512x256: FP64 (bit-identical) and FP32 over 300 steps;
* sphere channel, D3Q19 256x128x128: FP64 / FP32 / FP16 over 3 steps;
* sedimenting disc, D2Q9 135x1073 with a free disc: FP64 (bit-identical,
  trajectory included) and FP32 over 400 steps;
* 64-sphere box, D3Q19 512x256x256, FP32 -- exactly the benchmark's launch
  configuration: the force/torque of sampled moving spheres is checked
  against the oracle run on a periodic sub-box around each sphere.  The fluid
  starts at rest and information travels one cell per step, so for the first
  k steps an isolated sphere sees exactly the same flow in the sub-box as in
  the full box.
Measured errors are written to $LBM_PARITY_REPORT (a JSON file) when set.
"""
import numpy as np
import pytest

from parity_util import TOL_FP64_FT, TOL_RED_FT, TOL_RED_POP, ft_rel_error, pop_error, report

pytestmark = pytest.mark.gpu


_ORACLE_CACHE = {}


def _oracle_run(oracle_mod, spec, steps):
    """the oracle ignores the precision key: one run serves every mode"""
    key = (spec["name"], steps)
    if key not in _ORACLE_CACHE:
        ref = oracle_mod.Oracle(spec)
        ref.step(steps)
        _ORACLE_CACHE[key] = (ref.solid(), ref.fhat(), {k: ref.force_torque(k) for k in
                                                       ("static", "lattice", "moving")}, ref.series())
    return _ORACLE_CACHE[key]


def _report(key, value):
    report(key, value)


def test_channel_cylinder_full_5000_steps_fp64(oracle_mod):
    from paper_1407_4524_gb300 import lbm, workloads as W
    spec = W.channel_cylinder_2d("fp64")
    steps = spec["steps"]
    dom = lbm.Domain(spec, device=0)
    dom.step(steps)
    ref = oracle_mod.Oracle(spec)
    ref.step(steps)
    fl = ref.solid() < 0
    assert np.array_equal(dom.populations()[:, fl], ref.fhat()[:, fl])
    s_gpu, s_ref = dom.series(), ref.series()
    assert np.array_equal(s_gpu, s_ref)
    e = ft_rel_error(dom.force_torque("static"), ref.force_torque("static"), spec)
    assert e <= TOL_FP64_FT
    drag = s_ref[-1, 0, 0]
    _report("channel_cylinder_2d_fp64_5000", {"bitwise": True, "ft_rel": e, "drag_final": float(drag),
                                              "lift_final": float(s_ref[-1, 0, 1])})


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_moving_cylinders_full_size(oracle_mod, prec):
    from paper_1407_4524_gb300 import lbm, workloads as W
    spec = W.moving_cylinders_2d(prec)
    steps = 300
    dom = lbm.Domain(spec, device=0)
    dom.step(steps)
    solid, fhat, ft, series = _oracle_run(oracle_mod, spec, steps)
    assert np.array_equal(dom.solid(), solid)
    perr = pop_error(dom.populations(), fhat, solid)
    errs = {k: ft_rel_error(dom.force_torque(k), ft[k], spec) for k in ("static", "lattice", "moving")}
    _report(f"moving_cylinders_2d_{prec}_300", {"pop_abs": perr, **errs})
    if prec == "fp64":
        assert np.array_equal(dom.series(), series)
    else:
        tol_pop = TOL_RED_POP if prec == "fp32" else 2e-4
        tol_ft = TOL_RED_FT if prec == "fp32" else 2e-2
        assert perr <= tol_pop
        assert max(errs.values()) <= tol_ft


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_sphere_channel_full_size(oracle_mod, prec):
    from paper_1407_4524_gb300 import lbm, workloads as W
    spec = W.sphere_channel_3d(prec)
    steps = 3
    dom = lbm.Domain(spec, device=0)
    dom.step(steps)
    solid, fhat, ft, series = _oracle_run(oracle_mod, spec, steps)
    assert np.array_equal(dom.solid(), solid)
    perr = pop_error(dom.populations(), fhat, solid)
    e = ft_rel_error(dom.force_torque("static"), ft["static"], spec)
    _report(f"sphere_channel_3d_{prec}_3", {"pop_abs": perr, "static": e})
    if prec == "fp64":
        assert np.array_equal(dom.series(), series)
        assert perr == 0.0
    else:
        assert perr <= (TOL_RED_POP if prec == "fp32" else 2e-4)
        assert e <= (TOL_RED_FT if prec == "fp32" else 2e-2)


def _isolated_moving(bodies, n, k_steps, count=3):
    L = np.array(n, float)
    picks = []
    for i, b in enumerate(bodies):
        if not np.any(b["U"]):
            continue
        ok = True
        for j, o in enumerate(bodies):
            if j == i:
                continue
            d = np.array(b["X0"]) - np.array(o["X0"])
            d -= L * np.floor(d / L + 0.5)
            if np.linalg.norm(d) - b["R"] - o["R"] < 2 * k_steps + 16:
                ok = False
                break
        if ok:
            picks.append(i)
        if len(picks) == count:
            break
    return picks


def test_sphere_swarm_full_size_sampled(oracle_mod):
    """The benchmark configuration itself (512x256x256, 64 spheres, FP32)."""
    from paper_1407_4524_gb300 import lbm, workloads as W
    spec = W.sphere_swarm_3d("fp32")
    k = 4
    dom = lbm.Domain(spec, device=0)
    dom.step(k)
    picks = _isolated_moving(spec["bodies"], spec["n"], k)
    assert picks, "no isolated moving sphere to sample"
    out = {}
    for i in picks:
        b = dict(spec["bodies"][i])
        half = int(np.ceil(b["R"])) + 2 * k + 8
        m = 2 * half
        X = np.array(b["X0"])
        shift = np.floor(X) - half
        sub = dict(lattice="D3Q19", n=(m, m, m), tau=spec["tau"], precision="fp64",
                   bodies=[dict(b, X0=tuple(X - shift))])
        ref = oracle_mod.Oracle(sub)
        ref.step(k)
        errs = {}
        for kind in ("static", "lattice", "moving"):
            g = dom.force_torque(kind)[:, i:i + 1]
            r = ref.force_torque(kind)
            errs[kind] = ft_rel_error(g, r, spec, bodies=[i])
        out[str(i)] = errs
        assert max(errs.values()) <= TOL_RED_FT, (i, errs)
    _report("sphere_swarm_3d_fp32_sampled_4", out)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sedimenting_ellipse_full_size(oracle_mod, prec):
    """The paper's sedimenting ellipse (D2Q9 135x1676, free ellipse at 45
    degrees, r_rho = 1.10) over 300 steps: FP64 bit-identical, FP32 within
    tolerance."""
    from paper_1407_4524_gb300 import lbm, workloads as W
    spec = W.sedimenting_ellipse_2d(prec)
    steps = 300
    dom = lbm.Domain(spec, device=0)
    dom.step(steps)
    ref = oracle_mod.Oracle(spec)
    ref.step(steps)
    st, st_ref = dom.body_state(), ref.body_state()
    assert st_ref[0, 4] < 0 and st_ref[0, 8] != 0.0  # falls and turns
    if prec == "fp64":
        assert np.array_equal(dom.series(), ref.series())
        assert np.array_equal(st, st_ref)
        err = 0.0
    else:
        err = ft_rel_error(dom.force_torque("lattice"), ref.force_torque("lattice"), spec)
        assert err <= TOL_RED_FT
        assert np.abs(st[:, :3] - st_ref[:, :3]).max() <= 1e-6
    _report(f"sedimenting_ellipse_2d_{prec}_{steps}", {"lattice_ft_rel": err, "uy_final": float(st_ref[0, 4]),
                                                        "w_final": float(st_ref[0, 8])})


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sedimenting_disc_full_size(oracle_mod, prec):
    """The paper's sedimenting disc (D2Q9 135x1073, walls, free disc,
    r_rho = 1.01) over 400 steps: FP64 bit-identical series and trajectory;
    FP32 within tolerance."""
    from paper_1407_4524_gb300 import lbm, workloads as W
    spec = W.sedimenting_disc_2d(prec)
    steps = 400
    dom = lbm.Domain(spec, device=0)
    dom.step(steps)
    ref = oracle_mod.Oracle(spec)
    ref.step(steps)
    st, st_ref = dom.body_state(), ref.body_state()
    assert st_ref[0, 4] < 0  # it falls
    if prec == "fp64":
        assert np.array_equal(dom.series(), ref.series())
        assert np.array_equal(st, st_ref)
        err = 0.0
    else:
        err = ft_rel_error(dom.force_torque("lattice"), ref.force_torque("lattice"), spec)
        assert err <= TOL_RED_FT
        assert np.abs(st[:, :3] - st_ref[:, :3]).max() <= 1e-6
    _report(f"sedimenting_disc_2d_{prec}_{steps}", {"lattice_ft_rel": err, "uy_final": float(st_ref[0, 4]),
                                                     "dy": float(st_ref[0, 1] - spec["bodies"][0]["X0"][1])})
