"""GPU vs FP64 oracle at the benchmark configurations' full sizes.

* channel + cylinder, D2Q9 200x80, FP64, all 5000 steps: bit-identical
  populations and force/torque series;
* moving cylinders, D2Q9 512x256: FP64 (bit-identical), FP32 and FP16 over 1000 steps;
* sphere channel, D3Q19 256x128x128: FP64 (bit-identical) / FP32 / FP16 over 50 steps;
* sedimenting disc, D2Q9 135x1073 with a free disc: FP64 (bit-identical,
  trajectory included) and FP32 over 400 steps;
* 64-sphere box, D3Q19 512x256x256, FP32 and FP16, 50 steps -- exactly the
  benchmark's launch configuration: the force/torque of a moving and a static
  sphere and the populations around them are checked against the oracle run
  on a periodic sub-box that holds every body within their light cone
  (information moves at most one node per axis and step).
Measured errors are written to $LBM_PARITY_REPORT (a JSON file) when set.
"""
import numpy as np
import pytest

from parity_util import (TOL_FP16_FT, TOL_FP16_POP, TOL_FP64_FT, TOL_RED_FT, TOL_RED_POP, ft_rel_error,
                         pop_error, report)

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
    steps = 1000
    dom = lbm.Domain(spec, device=0)
    dom.step(steps)
    solid, fhat, ft, series = _oracle_run(oracle_mod, spec, steps)
    assert np.array_equal(dom.solid(), solid)
    perr = pop_error(dom.populations(), fhat, solid)
    errs = {k: ft_rel_error(dom.force_torque(k), ft[k], spec) for k in ("static", "lattice", "moving")}
    _report(f"moving_cylinders_2d_{prec}_{steps}", {"pop_abs": perr, **errs})
    if prec == "fp64":
        assert np.array_equal(dom.series(), series)
    else:
        tol_pop = TOL_RED_POP if prec == "fp32" else TOL_FP16_POP
        tol_ft = TOL_RED_FT if prec == "fp32" else TOL_FP16_FT
        assert perr <= tol_pop
        assert max(errs.values()) <= tol_ft


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_sphere_channel_full_size(oracle_mod, prec):
    from paper_1407_4524_gb300 import lbm, workloads as W
    spec = W.sphere_channel_3d(prec)
    steps = 50
    dom = lbm.Domain(spec, device=0)
    dom.step(steps)
    solid, fhat, ft, series = _oracle_run(oracle_mod, spec, steps)
    assert np.array_equal(dom.solid(), solid)
    perr = pop_error(dom.populations(), fhat, solid)
    e = ft_rel_error(dom.force_torque("static"), ft["static"], spec)
    _report(f"sphere_channel_3d_{prec}_{steps}", {"pop_abs": perr, "static": e})
    if prec == "fp64":
        assert np.array_equal(dom.series(), series)
        assert perr == 0.0
    else:
        assert perr <= (TOL_RED_POP if prec == "fp32" else TOL_FP16_POP)
        assert e <= (TOL_RED_FT if prec == "fp32" else TOL_FP16_FT)


def _mimg(d, L):
    return d - L * np.floor(d / L + 0.5)


def _subbox(spec, targets, k, margin=30):
    """A periodic sub-box of the (fully periodic) sphere-swarm box around the
    bodies `targets` in which their first k steps are exactly those of the
    full box.  Information moves at most one node per axis and step
    (|c_i|_inf = 1), so at step k a target's force and the populations near
    it depend only on what lies within Chebyshev distance k + 1.  The box is
    centred between the targets, with half-width H = (their reach) + k +
    margin; it holds every body that lies wholly inside it (at the same
    relative position), and the test asserts that every body it leaves out,
    and every periodic image of a body it holds, is more than k + 4 nodes
    from every target's surface (Chebyshev, swept positions included).
    Returns H, the integer shift (full node x -> sub-box node (x - shift)
    mod n), the indices of the bodies held and of those left out, and the
    sub-box positions of every body."""
    L = np.array(spec["n"], float)
    B = spec["bodies"]
    base = np.floor(np.array(B[targets[0]]["X0"]))
    d = [_mimg(np.array(b["X0"]) - base, L) for b in B]
    drift = [float(np.abs(np.array(b["U"])).max()) * k for b in B]
    c = np.floor(np.mean([d[t] for t in targets], axis=0))
    H = int(np.ceil(max(np.abs(d[t] - c).max() + B[t]["R"] + drift[t] for t in targets) + k + margin))
    m = 2 * H
    assert np.all(m <= L)
    shift = (base + c - H).astype(np.int64)
    pos = [d[i] - c + H for i in range(len(B))]
    held, left = [], []
    for i, b in enumerate(B):
        r = b["R"] + drift[i] + 2
        (held if np.all(pos[i] >= r) and np.all(pos[i] <= m - r) else left).append(i)
    for t in targets:
        assert t in held
        for q in left:
            gap = np.abs(_mimg(d[q] - d[t], L)).max() - B[q]["R"] - B[t]["R"] - drift[q] - drift[t]
            assert gap > k + 4, (t, q, gap)
        for p in held:
            gap = (m - np.abs(d[p] - d[t])).min() - B[p]["R"] - B[t]["R"] - drift[p] - drift[t]
            assert gap > k + 4, (t, p, gap)
    return H, shift, held, left, pos


def _exact_nodes(spec, H, held, left, pos, targets, k, reach=14):
    """Sub-box nodes near the targets (Chebyshev distance <= R + reach from a
    target's pose at step k) whose state at step k is the full box's: every
    body that differs between the two boxes (one left out, or a periodic
    image of one held) is more than k + 2 nodes from them.  Returns a boolean
    mask over the sub-box [z][y][x]."""
    L = np.array(spec["n"], float)
    B = spec["bodies"]
    m = 2 * H
    ax = np.arange(m, dtype=float)
    near = np.zeros((m, m, m), dtype=bool)
    for t in targets:
        X = pos[t] + k * np.array(B[t]["U"])
        r = B[t]["R"] + reach
        near |= ((np.abs(ax - X[2]) <= r)[:, None, None] & (np.abs(ax - X[1]) <= r)[None, :, None]
                 & (np.abs(ax - X[0]) <= r)[None, None, :])
    ok = near.copy()
    sources = []  # (centre in sub-box coordinates, period for the node displacement, reach)
    for q in left:
        sources.append((pos[q], L, B[q]["R"] + float(np.abs(np.array(B[q]["U"])).max()) * k))
    for p in held:
        for s in np.ndindex(3, 3, 3):
            if s == (1, 1, 1):
                continue
            sources.append((pos[p] + (np.array(s[::-1]) - 1) * m, None,
                            B[p]["R"] + float(np.abs(np.array(B[p]["U"])).max()) * k))
    for X, per, rq in sources:
        dx, dy, dz = ax - X[0], ax - X[1], ax - X[2]
        if per is not None:
            dx, dy, dz = _mimg(dx, per[0]), _mimg(dy, per[1]), _mimg(dz, per[2])
        cheb = np.maximum(np.maximum(np.abs(dz)[:, None, None], np.abs(dy)[None, :, None]),
                          np.abs(dx)[None, None, :])
        ok &= cheb - rq > k + 2
    return ok, near


def test_sphere_swarm_full_size_sampled(oracle_mod):
    """The benchmark configuration itself (512x256x256 periodic, 64 spheres,
    32 moving), 50 steps, FP32 and FP16, exactly the benchmark's launch
    configuration.  A moving sphere (13) and a static sphere next to it (48),
    each with moving neighbours within reach, are checked against the oracle
    run on a periodic 206^3 sub-box that holds every body within their light
    cone (see _subbox): all three force/torque forms of both bodies at every
    step, and the populations at step 50 on the nodes around them whose state
    the sub-box reproduces exactly (see _exact_nodes)."""
    from paper_1407_4524_gb300 import lbm, workloads as W
    k = 50
    targets = [13, 48]
    spec32 = W.sphere_swarm_3d("fp32")
    B = spec32["bodies"]
    assert np.any(B[13]["U"]) and not np.any(B[48]["U"])
    H, shift, held, left, pos = _subbox(spec32, targets, k)
    m = 2 * H
    sub = dict(lattice="D3Q19", n=(m, m, m), tau=spec32["tau"], precision="fp64",
               bodies=[dict(B[i], X0=tuple(pos[i])) for i in held])
    ref = oracle_mod.Oracle(sub)
    ref.step(k)
    f_ref = ref.fhat()
    solid_ref = ref.solid()
    ft_ref = {kind: ref.force_torque(kind) for kind in ("static", "lattice", "moving")}
    del ref
    ok, near = _exact_nodes(spec32, H, held, left, pos, targets, k)
    fluid = ok & (solid_ref < 0)
    assert fluid.sum() > 0.5 * (near & (solid_ref < 0)).sum()  # most of the region around the targets
    n = spec32["n"]
    idx = [(np.arange(m) + shift[a]) % n[a] for a in range(3)]
    out = {}
    for prec in ("fp32", "fp16"):
        dom = lbm.Domain(W.sphere_swarm_3d(prec), device=0)
        dom.step(k)
        errs = {}
        for j, t in enumerate(targets):
            for kind in ("static", "lattice", "moving"):
                g = dom.force_torque(kind)[:, t:t + 1]
                r = ft_ref[kind][:, held.index(t):held.index(t) + 1]
                errs[f"{t}/{kind}"] = ft_rel_error(g, r, spec32, bodies=[t])
        sol = dom.solid()[np.ix_(idx[2], idx[1], idx[0])]
        assert np.array_equal(sol[near] < 0, solid_ref[near] < 0)
        f_gpu = dom.populations()[:, idx[2][:, None, None], idx[1][None, :, None], idx[0][None, None, :]]
        dom.close()
        perr = float(np.abs(f_gpu[:, fluid] - f_ref[:, fluid]).max())
        del f_gpu
        out[prec] = {"pop_abs": perr, "nodes": int(fluid.sum()), **errs}
        tol_pop = TOL_RED_POP if prec == "fp32" else TOL_FP16_POP
        tol_ft = TOL_RED_FT if prec == "fp32" else TOL_FP16_FT
        assert perr <= tol_pop, (prec, perr)
        assert max(errs.values()) <= tol_ft, (prec, errs)
    _report("sphere_swarm_3d_sampled_50", out)


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
