"""Short-time noise of the force series by force form and refill rule.

The force discussion of Sec. 3 (after Eq. ForceInMovement) names the
impulsive A+ / A- terms of the lattice-frame force as the main source of its
short-time noise, which the moving-frame form (Eq.
ForceInMovementMovingFrame) avoids, and states that the extrapolation and
the u_B-equilibrium refill of uncovered nodes give less noise than the
equilibrium from neighbour averages.  ``force_noise`` runs one problem on the
GPU under each refill rule and reports, per rule and form, the noise of one
force component of one body: the standard deviation of the series minus its centred
moving average (``window`` steps), after ``skip`` transient steps.
"""
from __future__ import annotations

import numpy as np

from . import lbm

RULES = ("uB", "ubar", "extrap")


def noise(series, window: int = 21, skip: int = 0) -> float:
    F = np.asarray(series[skip:], float)
    ma = np.convolve(F, np.ones(window) / window, mode="same")
    h = window // 2
    return float(np.std((F - ma)[h:len(F) - h]))


def force_noise(spec: dict, steps: int, body: int = 0, component: int = 0, window: int = 21,
                skip: int | None = None, rules=RULES, device: int = 0) -> dict:
    """{rule: {"lattice", "moving", "static" (noise of force component
    `component`), "drag" (its mean in the lattice frame), "extrapolated"
    (uncovered nodes refilled by extrapolation)}}."""
    if skip is None:
        skip = steps // 4
    out = {}
    for rule in rules:
        dom = lbm.Domain(dict(spec, refill=rule), device=device, series_capacity=steps)
        try:
            dom.step(steps)
            s = dom.force_torque("static")[:, body, component]
            lat = dom.force_torque("lattice")[:, body, component]
            mv = dom.force_torque("moving")[:, body, component]
            out[rule] = {"lattice": noise(lat, window, skip), "moving": noise(mv, window, skip),
                         "static": noise(s, window, skip), "drag": float(np.mean(lat[skip:])),
                         "extrapolated": dom.stats()["extrapolated"]}
        finally:
            dom.close()
    return out


def main(argv=None):
    """python -m paper_1407_4524_gb300.noise: the x force of the translating
    cylinder of the moving-cylinders workload (512 x 256 D2Q9, R = 12 at
    U = 0.02), or the y force of the sedimenting disc."""
    import argparse
    import json

    from . import workloads
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="moving_cylinders_2d", choices=["moving_cylinders_2d", "sedimenting_disc_2d"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "fp16"])
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--window", type=int, default=21)
    args = ap.parse_args(argv)
    spec = getattr(workloads, args.workload)(precision=args.precision)
    steps = int(args.steps or spec["steps"])
    comp = 1 if args.workload == "sedimenting_disc_2d" else 0
    res = force_noise(spec, steps, component=comp, window=args.window)
    print(json.dumps({"workload": args.workload, "precision": args.precision, "steps": steps,
                      "window": args.window, "component": "xy"[comp], "noise": res}))


if __name__ == "__main__":
    main()
