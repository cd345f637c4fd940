"""Helpers shared by the GPU parity tests (comparison metrics only)."""
import numpy as np

# tolerances of the method's precision modes: FP64 mode 1e-12 relative on force and
# torque; reduced precision 1e-5 absolute on populations (rho ~ 1) and 1e-4
# relative on force and torque after N steps.
TOL_FP64_FT = 1e-12
TOL_FP64_POP = 1e-13
TOL_RED_POP = 1e-5
TOL_RED_FT = 1e-4


def char_scales(spec):
    """Characteristic force and torque of each body: F_c = rho0 U^2 R^(D-1)
    with U the largest of the inflow, the initial flow and the body's surface
    speed |U| + |W| R; T_c = F_c R.  Used as a floor of the relative-error
    denominator, so that a force that vanishes by symmetry (or because the
    fluid around the body is still at rest) is compared with the problem's
    force scale instead of with its own round-off."""
    D = 2 if spec["lattice"] == "D2Q9" else 3
    rho0 = spec.get("rho0", 1.0)
    u_flow = max(abs(spec.get("inlet", {}).get("u", 0.0)),
                 float(np.linalg.norm(spec.get("u0", (0.0, 0.0, 0.0)))))
    out = []
    for b in spec.get("bodies", []):
        W = b.get("W", 0.0)
        wn = abs(W) if np.isscalar(W) else float(np.linalg.norm(W))
        ub = float(np.linalg.norm(b.get("U", (0.0, 0.0, 0.0)))) + wn * b["R"]
        U = max(u_flow, ub, 1e-3)
        fc = rho0 * U * U * b["R"] ** (D - 1)
        out.append((fc, fc * b["R"]))
    return out


def ft_rel_error(ft, ref, spec=None, bodies=None):
    """Normwise relative error per body: max over steps and components of
    |ft - ref|, divided by the largest |ref| component of that body's force
    (first three) or torque (last three) series -- or by the body's
    characteristic scale when that is larger (see char_scales); returns the
    max over bodies and over force/torque."""
    ft = np.asarray(ft)
    ref = np.asarray(ref)
    assert ft.shape == ref.shape, (ft.shape, ref.shape)
    floors = char_scales(spec) if spec is not None else None
    if floors is not None and bodies is not None:
        floors = [floors[i] for i in bodies]
    worst = 0.0
    for b in range(ref.shape[1]):
        for k, sl in enumerate((slice(0, 3), slice(3, 6))):
            scale = np.abs(ref[:, b, sl]).max()
            if floors is not None:
                scale = max(scale, floors[b][k])
            err = np.abs(ft[:, b, sl] - ref[:, b, sl]).max()
            rel = err / scale if scale > 0.0 else err
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
