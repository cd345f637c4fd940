"""Invariants checked on the GPU's own outputs, independently of the oracle:
in a periodic box with moving bodies the fluid's momentum changes by exactly
minus the bodies' lattice-frame force (Eq. ForceInMovement: the static link
sum plus the impulsive terms of the covered and uncovered nodes), step by
step, in the FP64 mode -- the discrete Reynolds-transport balance of Sec. 3."""
import numpy as np
import pytest

from test_parity_gpu import CASES_2D, CASES_3D

pytestmark = pytest.mark.gpu


def _fluid_momentum(dom, c):
    """sum over fluid nodes of sum_i c_i fhat_i (collision conserves it)"""
    f = dom.populations().reshape(dom.q, -1)
    fluid = dom.solid().reshape(-1) < 0
    return (c.T @ f[:, fluid]).sum(1)


@pytest.mark.parametrize("dim,name", [("2d", "moving_cylinders_periodic"), ("3d", "moving_spheres_periodic")])
def test_momentum_balance_with_moving_bodies(dim, name):
    from paper_1407_4524_gb300 import lbm
    spec = dict((CASES_2D if dim == "2d" else CASES_3D)[name], precision="fp64")
    dom = lbm.Domain(spec, device=0)
    c, _, _ = lbm.lbm_lattice_table(dom.q)
    c = c.astype(float)
    P0 = _fluid_momentum(dom, c)
    worst, scale, impulsive = 0.0, 0.0, 0
    for _ in range(20):
        t = dom.t
        dom.step(1)
        P1 = _fluid_momentum(dom, c)
        F = dom.force_torque("lattice", first=t, count=1)[0, :, :3].sum(0)
        imp = dom.force_torque("impulsive", first=t, count=1)[0, :, :3]
        impulsive += int(np.abs(imp).max() > 0)
        worst = max(worst, np.abs(P1 - P0 + F).max())
        scale = max(scale, np.abs(F).max())
        P0 = P1
    dom.close()
    assert scale > 1e-3 and impulsive > 3
    assert worst <= 1e-12 * scale, (worst, scale)
