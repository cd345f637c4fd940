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
