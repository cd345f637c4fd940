"""Seeded workload generators (no GPU): determinism, ranges, and that the
served requests satisfy the library's body-placement rules."""
import numpy as np

from paper_1407_4524_gb300 import workloads as W


def test_serving_trace_seeded_and_in_range():
    a = W.serving_trace(n_requests=50)
    b = W.serving_trace(n_requests=50)
    assert [r["arrival_s"] for r in a] == [r["arrival_s"] for r in b]
    gaps = np.diff([0.0] + [r["arrival_s"] for r in a])
    assert np.all(gaps > 0)
    for r in a:
        assert 0.52 <= r["tau"] <= 1.0
        assert 0.01 <= r["inlet"]["u"] <= 0.05
        assert 2000 <= r["steps"] <= 20000
        assert len(r["bodies"]) == 1
        R = r["bodies"][0]["R"]
        assert 5.0 <= R <= 15.0
        n = r["n"]
        if r["lattice"] == "D2Q9":
            assert tuple(n) in W.SERVING_D2Q9_SIZES
        else:
            assert tuple(n) in W.SERVING_D3Q19_SIZES
        X = r["bodies"][0]["X0"]
        # 3 cells from the non-periodic x faces (and y walls in 2-D)
        assert X[0] - R >= 3.0 and X[0] + R <= n[0] - 4.0
        if r["lattice"] == "D2Q9":
            assert X[1] - R >= 3.0 and X[1] + R <= n[1] - 4.0
        else:
            assert 2 * R + 4 < min(n[1], n[2])


def test_sphere_swarm_gap_rule():
    spec = W.sphere_swarm_3d(n=(128, 96, 96), n_bodies=12, steps=200)
    L = np.array(spec["n"], dtype=float)
    bs = spec["bodies"]
    assert len(bs) == 12
    for i in range(len(bs)):
        for j in range(i):
            d = np.array(bs[i]["X0"]) - np.array(bs[j]["X0"])
            d -= L * np.floor(d / L + 0.5)
            assert np.linalg.norm(d) - bs[i]["R"] - bs[j]["R"] >= 2.0
    assert all(np.linalg.norm(b["U"]) == 0.0 for b in bs[0::2])
    assert all(np.linalg.norm(b["U"]) <= 0.02 for b in bs[1::2])


def _golden_setup():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "sedimentation_setup.txt")
    out = {}
    for line in open(path):
        line = line.split("#")[0].split()
        if line:
            vals = [float(v) if v[0].isdigit() else v for v in line[1:]]
            out[line[0]] = vals if len(vals) > 1 else vals[0]
    return out


def test_sedimentation_workloads_follow_the_printed_setup():
    """The sedimentation workloads in lattice units restate the paper's
    printed set-up: lattice size, tau, the on-node walls of the Zou-He edges
    spanning the channel (and the printed sizes agree: (ny - 1) dx = H),
    body sizes, start positions, orientation, density ratios, and gravity
    through dt = nu_lattice dx^2 / nu."""
    import math
    G = _golden_setup()
    nu_l = (G["tau"] - 0.5) / 3.0
    # disc
    nx, ny = (int(v) for v in G["disc.n"])
    d = G["disc.d"]
    width = G["disc.W_over_d"] * d
    dx = width / (nx - 1)
    assert abs((ny - 1) * dx - G["disc.H_over_W"] * width) < 1e-12
    dt = nu_l * dx * dx / G["nu"]
    for r_rho in G["disc.r_rho"]:
        spec = W.sedimenting_disc_2d(density_ratio=r_rho)
        assert spec["lattice"] == G["lattice"] and tuple(spec["n"]) == (nx, ny) and spec["tau"] == G["tau"]
        b = spec["bodies"][0]
        assert b["shape"] == "cylinder" and b["free"] and b["density_ratio"] == r_rho
        assert math.isclose(b["R"], 0.5 * d / dx, rel_tol=1e-12)
        x_c, y_c = G["disc.centre"]
        assert math.isclose(b["X0"][0], 0.5 * (nx - 1) + x_c / dx, rel_tol=1e-12)
        assert math.isclose(b["X0"][1], (G["disc.origin_above_bottom"] + y_c) / dx, rel_tol=1e-12)
        assert math.isclose(-spec["gravity"][1], G["g"] * dt * dt / dx, rel_tol=1e-12)
    # ellipse
    nx, ny = (int(v) for v in G["ellipse.n"])
    a = G["ellipse.a"]
    width = G["ellipse.blockage"] * a
    dx = width / (nx - 1)
    assert abs((ny - 1) * dx - G["ellipse.H_over_a"] * a) < 1e-12
    dt = nu_l * dx * dx / G["nu"]
    spec = W.sedimenting_ellipse_2d()
    assert tuple(spec["n"]) == (nx, ny) and spec["tau"] == G["tau"]
    b = spec["bodies"][0]
    assert b["shape"] == "ellipse" and b["free"] and b["density_ratio"] == G["ellipse.r_rho"]
    assert math.isclose(b["R"], 0.5 * a / dx, rel_tol=1e-12)
    assert math.isclose(b["R2"], 0.5 * a / G["ellipse.aspect"] / dx, rel_tol=1e-12)
    assert math.isclose(b["theta0"], G["ellipse.theta0_over_pi"] * math.pi, rel_tol=1e-15)
    cx, cy = G["ellipse.centre_over_W"]
    assert math.isclose(b["X0"][0], cx * (nx - 1), rel_tol=1e-12)
    assert math.isclose(b["X0"][1], (G["ellipse.origin_above_bottom"] + cy) / dx, rel_tol=1e-12)
    assert math.isclose(-spec["gravity"][1], G["g"] * dt * dt / dx, rel_tol=1e-12)
