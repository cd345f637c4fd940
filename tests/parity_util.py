"""Helpers shared by the GPU parity tests (comparison metrics only)."""
import numpy as np

# tolerances of the method's precision modes: FP64 mode 1e-12 relative on force and
# torque; reduced precision 1e-5 absolute on populations (rho ~ 1) and 1e-4
# relative on force and torque after N steps.
TOL_FP64_FT = 1e-12
TOL_FP64_POP = 1e-13
TOL_RED_POP = 1e-5
TOL_RED_FT = 1e-4
# FP16 storage of f - w is outside that tolerance by its format: 11
# significant bits put the rounding of a stored deviation of 0.03-0.06 alone
# at up to 1.5e-5, and the error after N steps scales with the storage ulp
# (13-14 significant bits are needed).  Its tests assert these bounds (the
# largest errors measured are 4.5e-5 and 5.4e-4) and report the errors.
TOL_FP16_POP = 1e-4
TOL_FP16_FT = 2e-3


# a body's wrench series (below) that stays under this fraction of its
# characteristic force vanishes: zero by symmetry (or because the fluid near
# the body is at rest) up to FP64 round-off
VANISHING = 1e-9


def char_scales(spec):
    """Characteristic force and torque of each body: F_c = rho0 U^2 R^(D-1)
    with U the largest of the inflow, the initial flow and the body's surface
    speed |U| + |W| R; T_c = F_c R.  Only the error of a series that vanishes
    in the oracle is measured against this scale (see ft_rel_error)."""
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
    """Normwise relative error of each body's wrench series, maximum over
    bodies.  The wrench of a body at step t is (F, T / R), R its radius (the
    first semi-axis of an ellipse): the torque is a sum of link momenta with
    lever arms up to R, so T / R has the units and the round-off scale of a
    force.  Error = max over steps and the six components of |w - w_oracle|,
    divided by the oracle's maximum over steps and components of |w_oracle|
    -- the series-maximum normalisation of the force and torque series, taken
    over the wrench so that a torque that nearly cancels (much smaller than R
    times the force) is not measured against its own round-off.  A body whose
    oracle wrench vanishes (below VANISHING times F_c: zero by symmetry) is
    measured against F_c instead.  Without a problem description the force
    and the torque series are each normalised by their own maximum."""
    ft = np.asarray(ft)
    ref = np.asarray(ref)
    assert ft.shape == ref.shape, (ft.shape, ref.shape)
    if ref.shape[0] == 0:
        return 0.0
    if spec is None:
        worst = 0.0
        for b in range(ref.shape[1]):
            for sl in (slice(0, 3), slice(3, 6)):
                scale = np.abs(ref[:, b, sl]).max()
                err = np.abs(ft[:, b, sl] - ref[:, b, sl]).max()
                worst = max(worst, err / scale if scale > 0.0 else err)
        return worst
    idx = list(range(len(spec["bodies"]))) if bodies is None else list(bodies)
    floors = char_scales(spec)
    worst = 0.0
    for j, bi in enumerate(idx):
        R = float(spec["bodies"][bi]["R"])
        w_ref = np.concatenate([ref[:, j, 0:3], ref[:, j, 3:6] / R], axis=1)
        w = np.concatenate([ft[:, j, 0:3], ft[:, j, 3:6] / R], axis=1)
        scale = np.abs(w_ref).max()
        if scale < VANISHING * floors[bi][0]:
            scale = floors[bi][0]
        worst = max(worst, np.abs(w - w_ref).max() / scale)
    return worst


def ft_series_errors(ft, ref):
    """Per body, the force and the torque error each relative to its own
    series maximum (reported beside ft_rel_error; a series that is tiny or
    zero gives a large or infinite value here)."""
    ft = np.asarray(ft)
    ref = np.asarray(ref)
    out = []
    for b in range(ref.shape[1]):
        row = []
        for sl in (slice(0, 3), slice(3, 6)):
            scale = np.abs(ref[:, b, sl]).max() if ref.shape[0] else 0.0
            err = np.abs(ft[:, b, sl] - ref[:, b, sl]).max() if ref.shape[0] else 0.0
            row.append(float(err / scale) if scale > 0.0 else (0.0 if err == 0.0 else float("inf")))
        out.append(row)
    return out


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
