"""Helpers shared by the GPU parity tests (comparison metrics only)."""
import numpy as np

# tolerances (BASELINE the benchmark spec): FP64 mode 1e-12 relative on force and
# torque; reduced precision 1e-5 absolute on populations (rho ~ 1) and 1e-4
# relative on force and torque after N steps.
TOL_FP64_FT = 1e-12
TOL_FP64_POP = 1e-13
TOL_RED_POP = 1e-5
TOL_RED_FT = 1e-4


def ft_rel_error(ft, ref):
    """Normwise relative error per body: max over steps and components of
    |ft - ref|, divided by the largest |ref| component of that body's force
    (first three) or torque (last three) series; returns the max over bodies
    and over force/torque."""
    ft = np.asarray(ft)
    ref = np.asarray(ref)
    assert ft.shape == ref.shape, (ft.shape, ref.shape)
    worst = 0.0
    for b in range(ref.shape[1]):
        for sl in (slice(0, 3), slice(3, 6)):
            scale = np.abs(ref[:, b, sl]).max()
            err = np.abs(ft[:, b, sl] - ref[:, b, sl]).max()
            if scale == 0.0:
                rel = err
            else:
                rel = err / scale
            worst = max(worst, rel)
    return worst


def pop_error(f_gpu, f_ref, solid):
    fluid = solid < 0
    return float(np.abs(f_gpu[:, fluid] - f_ref[:, fluid]).max())


def report(key, value):
    """append a measured error to the JSON file named by $LBM_PARITY_REPORT"""
    import json
    import os
    path = os.environ.get("LBM_PARITY_REPORT")
    if not path:
        return
    data = {}
    if os.path.exists(path):
        with open(path) as fh:
            data = json.load(fh)
    data[key] = value
    with open(path, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
