"""Pins of the oracle's free bodies (CPU only): Newton's equation integrated by
forward Euler from the lattice-frame force of each step (Eqs.
ForceInMovement / TorqueInMovement) with weight less buoyancy.

* from rest in fluid at rest the first step adds exactly (rho_b - rho0)/rho_b g
  to the velocity, the position follows with one step of delay;
* in a closed periodic box without gravity the fluid momentum plus the body's
  M U is conserved to round-off (this pins the sign of the force applied to the
  body, the force form -- static plus impulsive -- and that the pose advanced
  with the velocity the A+/A- sets were built from);
* a free cylinder, ellipse or sphere spinning at the centre of a closed box:
  the angular momentum of fluid plus body plus walls is conserved to
  round-off (pins the moments of inertia and the sign of the applied torque).
"""
import numpy as np
import pytest

from test_oracle_wall import _closed_box, _fluid_momentum, _tables


def _free(lat, U, W, r, shape_kw):
    b = dict(shape_kw, U=U, W=W, free=True, density_ratio=r)
    return b


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_first_step_from_rest(oracle_mod, lat):
    r = 1.7
    if lat == "D2Q9":
        g = (0.0, -2e-4, 0.0)
        spec = dict(lattice=lat, n=(40, 36), tau=0.8, gravity=g,
                    bodies=[dict(shape="cylinder", R=6.3, X0=(19.2, 17.6), free=True, density_ratio=r)])
    else:
        g = (1e-4, -2e-4, 5e-5)
        spec = dict(lattice=lat, n=(22, 20, 18), tau=0.8, gravity=g,
                    bodies=[dict(shape="sphere", R=4.4, X0=(10.6, 9.3, 8.8), free=True, density_ratio=r)])
    o = oracle_mod.Oracle(spec)
    s0 = o.body_state()[0]
    o.step(1)
    s1 = o.body_state()[0]
    F = o.force_torque("lattice")[0, 0, :3]
    assert np.abs(F).max() < 1e-13  # fluid at rest, body at rest
    assert np.array_equal(s1[:3], s0[:3])  # X(1) = X(0) + U(0) = X(0)
    expect = (r - 1.0) / r * np.array(g)
    assert np.allclose(s1[3:6], expect, rtol=1e-12, atol=1e-18)
    o.step(1)
    s2 = o.body_state()[0]
    assert np.allclose(s2[:3], s1[:3] + s1[3:6], rtol=0, atol=1e-15)  # X(2) = X(1) + U(1)


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_momentum_of_fluid_plus_body_is_conserved(oracle_mod, lat):
    r = 1.3
    if lat == "D2Q9":
        b = [dict(shape="cylinder", R=5.6, X0=(14.2, 13.7), U=(0.06, -0.04), W=(0.0, 0.0, 0.004),
                  free=True, density_ratio=r)]
        u0 = (0.0, 0.0)
        V = np.pi * 5.6 ** 2
    else:
        b = [dict(shape="sphere", R=4.1, X0=(8.2, 7.6, 7.3), U=(0.05, -0.03, 0.04),
                  W=(0.003, -0.002, 0.004), free=True, density_ratio=r)]
        u0 = (0.0, 0.0, 0.0)
        V = 4.0 / 3.0 * np.pi * 4.1 ** 3
    o = oracle_mod.Oracle(_closed_box(lat, b, u0))
    c, _, _ = _tables(oracle_mod, o)
    M = r * 1.0 * V
    P_fl, _, _ = _fluid_momentum(o, c)
    total0 = P_fl + M * o.body_state()[0, 3:6]
    err, scale, n_imp = 0.0, 0.0, 0
    U_first = o.body_state()[0, 3:6].copy()
    wall = np.zeros(3)  # momentum given to the box walls so far (their link force, summed over steps)
    for t in range(40):
        o.step(1)
        wall += o.edge_me()[:3]
        P_fl, _, _ = _fluid_momentum(o, c)
        total = P_fl + M * o.body_state()[0, 3:6] + wall
        err = max(err, np.abs(total - total0).max())
        row = o.series()[-1, 0]
        scale = max(scale, np.abs(row[0:3] + row[6:9]).max())
        n_imp += int(np.abs(row[6:9]).max() > 0)
    assert n_imp > 3
    assert scale > 0
    # the body has slowed down against the fluid, and the momentum it lost is in the fluid
    assert np.linalg.norm(o.body_state()[0, 3:6]) < np.linalg.norm(U_first)
    assert err <= 1e-12 * M * np.abs(U_first).max()


@pytest.mark.parametrize("shape", ["cylinder", "ellipse", "sphere"])
def test_angular_momentum_of_fluid_plus_spinning_body_is_conserved(oracle_mod, shape):
    """A free body spun up at the centre of a closed box, fluid at rest: box
    and body are symmetric under inversion through the centre, so the force
    stays zero and the body stays put, and the fluid's angular momentum plus
    the body's I W plus the torque given to the walls is conserved to
    round-off.  This pins the moment of inertia (M R^2 / 2, M (a^2 + b^2) / 4,
    2/5 M R^2 with M = rho_b V) and the sign of the torque applied to the body;
    the ellipse adds the impulsive terms of the nodes its rotation covers and
    uncovers (Eq. TorqueInMovement)."""
    r = 1.4
    if shape == "sphere":
        lat, R, R2 = "D3Q19", 4.3, None
        X0 = (8.5, 7.5, 7.0)  # centre of the 18 x 16 x 15 box
        W0 = np.array([0.003, -0.002, 0.004])
        b = dict(shape=shape, R=R, X0=X0, W=tuple(W0), free=True, density_ratio=r)
        M = r * 4.0 / 3.0 * np.pi * R ** 3
        I = 0.4 * M * R * R
    else:
        lat = "D2Q9"
        X0 = (16.5, 14.5)  # centre of the 34 x 30 box
        W0 = np.array([0.0, 0.0, 0.006])
        if shape == "cylinder":
            R, R2 = 5.7, None
            b = dict(shape=shape, R=R, X0=X0, W=W0[2], free=True, density_ratio=r)
            M = r * np.pi * R * R
            I = 0.5 * M * R * R
        else:
            R, R2 = 8.2, 4.6
            r, W0 = 3.0, np.array([0.0, 0.0, 0.012])  # heavier and faster: it keeps turning over nodes
            b = dict(shape=shape, R=R, R2=R2, theta0=0.35, X0=X0, W=W0[2], free=True, density_ratio=r)
            M = r * np.pi * R * R2
            I = 0.25 * M * (R * R + R2 * R2)
    o = oracle_mod.Oracle(_closed_box(lat, [b], (0.0,) * (2 if lat == "D2Q9" else 3)))
    c, _, _ = _tables(oracle_mod, o)

    def body_L(s, inertia):
        X, U, W = s[0:3], s[3:6], s[6:9]
        return inertia * W + np.cross(X, M * U)

    _, L_fl, _ = _fluid_momentum(o, c)
    total0 = L_fl + body_L(o.body_state()[0], I)
    total0_wrong = L_fl + body_L(o.body_state()[0], 2.0 * I)
    walls = np.zeros(3)
    err, err_wrong, n_imp = 0.0, 0.0, 0
    for _ in range(40):
        o.step(1)
        walls += o.edge_me()[3:]
        _, L_fl, _ = _fluid_momentum(o, c)
        s = o.body_state()[0]
        err = max(err, np.abs(L_fl + body_L(s, I) + walls - total0).max())
        err_wrong = max(err_wrong, np.abs(L_fl + body_L(s, 2.0 * I) + walls - total0_wrong).max())
        n_imp += int(np.abs(o.series()[-1, 0, 9:12]).max() > 0)
        assert np.abs(s[3:6]).max() < 1e-14  # no force: the body does not translate
    s = o.body_state()[0]
    spun_down = np.abs(s[6:9] - W0).max()
    assert spun_down > 1e-3 * np.abs(W0).max()  # the fluid took up a visible part of the spin
    assert err <= 1e-11 * I * np.abs(W0).max()
    assert err_wrong > 1e3 * err  # a wrong moment of inertia breaks the balance
    if shape == "ellipse":
        assert n_imp > 3
