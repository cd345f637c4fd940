"""Force-noise comparison on the GPU (refill rules x force forms), checked
against the same comparison run by the FP64 oracle on a small case."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_gpu_noise_matches_oracle_small_case(oracle_mod):
    from paper_1407_4524_gb300 import noise
    spec = dict(lattice="D2Q9", n=(120, 61), tau=0.6, edges={"x": "periodic", "y": ("wall", "wall")},
                bodies=[dict(shape="cylinder", R=6.4, X0=(30.3, 30.37), U=(0.05, 0.0))], precision="fp64")
    steps = 400
    res = noise.force_noise(spec, steps, window=21, skip=100)
    for rule, r in res.items():
        o = oracle_mod.Oracle(dict(spec, refill=rule))
        o.step(steps)
        lat = o.force_torque("lattice")[:, 0, 0]
        mv = o.force_torque("moving")[:, 0, 0]
        assert abs(r["lattice"] - noise.noise(lat, 21, 100)) <= 1e-12 * r["lattice"]
        assert abs(r["moving"] - noise.noise(mv, 21, 100)) <= 1e-12 * r["moving"]
        assert r["moving"] < 0.2 * r["lattice"]
        assert (r["extrapolated"] > 0) == (rule == "extrap")
        assert r["extrapolated"] == (o.extrapolated() if rule == "extrap" else 0)


def test_gpu_noise_full_workload():
    """The translating cylinder of the 512 x 256 moving-cylinders workload,
    FP32, 20000 steps: the moving-frame form is quieter than the lattice frame
    under every rule."""
    from paper_1407_4524_gb300 import noise, workloads
    spec = workloads.moving_cylinders_2d(precision="fp32")
    res = noise.force_noise(spec, int(spec["steps"]))
    for rule, r in res.items():
        assert np.isfinite(r["drag"]) and r["drag"] < 0.0
        assert r["moving"] < 0.5 * r["lattice"], (rule, r)
