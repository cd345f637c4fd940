"""Pins of the oracle's elliptic bodies (CPU only).

* its own sin / cos agree with the C library's to an ulp or two;
* an ellipse with equal semi-axes is the circle: same solid set, link set and
  (to round-off) the same Delta and force;
* every cut link's wall point x_F - Delta c_i lies on the ellipse, and the
  fluid side of it does not (checked against the ellipse equation);
* the solid set of a rotated ellipse covers about pi R R2 nodes and is
  unchanged by a rotation through pi;
* a rotating ellipse (which covers and uncovers nodes without translating)
  keeps the closed-box momentum balance exact with the A+/A- terms.
"""
import math

import numpy as np
import pytest

from test_oracle_wall import _closed_box, _fluid_momentum, _tables


def test_sincos_matches_libm(oracle_mod):
    xs = np.concatenate([np.linspace(-60.0, 60.0, 2001), [0.0, 1e-9, -1e-9, math.pi / 4, math.pi / 2, math.pi]])
    for x in xs:
        s, c = oracle_mod.sincos(x)
        assert abs(s - math.sin(x)) <= 4e-16 * max(1.0, abs(x) / 8)
        assert abs(c - math.cos(x)) <= 4e-16 * max(1.0, abs(x) / 8)


def test_equal_axes_is_the_circle(oracle_mod):
    base = dict(lattice="D2Q9", n=(40, 36), tau=0.7, u0=(0.03, 0.01))
    circ = oracle_mod.Oracle(dict(base, bodies=[dict(shape="cylinder", R=7.3, X0=(19.4, 17.2))]))
    ell = oracle_mod.Oracle(dict(base, bodies=[dict(shape="ellipse", R=7.3, R2=7.3, theta0=0.7, X0=(19.4, 17.2))]))
    assert np.array_equal(circ.solid(), ell.solid())
    c1, d1, e1 = circ.links(0)
    c2, d2, e2 = ell.links(0)
    assert np.array_equal(c1, c2) and np.array_equal(d1, d2)
    assert np.abs(e1 - e2).max() < 1e-13
    circ.step(20)
    ell.step(20)
    F1, F2 = circ.force_torque("static"), ell.force_torque("static")
    assert np.abs(F1 - F2).max() <= 1e-11 * np.abs(F1).max()


@pytest.mark.parametrize("theta0", [0.0, 0.4, 1.1, 2.9])
def test_link_deltas_lie_on_the_ellipse(oracle_mod, theta0):
    a, b = 8.3, 4.1
    X = np.array([20.6, 18.3])
    o = oracle_mod.Oracle(dict(lattice="D2Q9", n=(42, 38), tau=0.7,
                               bodies=[dict(shape="ellipse", R=a, R2=b, theta0=theta0, X0=tuple(X))]))
    c, _, _ = _tables(oracle_mod, o)
    cells, dirs, deltas = o.links(0)
    assert len(cells) > 40
    co, si = math.cos(theta0), math.sin(theta0)

    def q(p):
        d = p - X
        xi, eta = co * d[0] + si * d[1], co * d[1] - si * d[0]
        return (xi / a) ** 2 + (eta / b) ** 2

    nx = o.shape[0]
    for cell, i, dl in zip(cells, dirs, deltas):
        xf = np.array([cell % nx, cell // nx], dtype=float)
        ci = c[i][:2].astype(float)
        assert 0.0 < dl <= 1.0
        assert abs(q(xf - dl * ci) - 1.0) < 1e-12
        assert q(xf) > 1.0 and q(xf - ci) <= 1.0 + 1e-12


def test_solid_area_and_half_turn(oracle_mod):
    a, b = 11.2, 5.3
    spec = dict(lattice="D2Q9", n=(48, 44), tau=0.7)
    o1 = oracle_mod.Oracle(dict(spec, bodies=[dict(shape="ellipse", R=a, R2=b, theta0=0.6, X0=(23.5, 21.5))]))
    o2 = oracle_mod.Oracle(dict(spec, bodies=[dict(shape="ellipse", R=a, R2=b, theta0=0.6 + math.pi,
                                                    X0=(23.5, 21.5))]))
    n1 = (o1.solid() >= 0).sum()
    perimeter = math.pi * (3 * (a + b) - math.sqrt((3 * a + b) * (a + 3 * b)))
    assert abs(n1 - math.pi * a * b) < 0.5 * perimeter
    assert np.array_equal(o1.solid(), o2.solid())


def test_rotating_ellipse_closed_box_balance(oracle_mod):
    b = [dict(shape="ellipse", R=7.6, R2=3.9, theta0=0.3, X0=(16.7, 15.2), W=0.01)]
    o = oracle_mod.Oracle(_closed_box("D2Q9", b, (0.0, 0.0)))
    c, _, _ = _tables(oracle_mod, o)
    P0, _, _ = _fluid_momentum(o, c)
    err, scale, n_imp = 0.0, 0.0, 0
    for t in range(40):
        o.step(1)
        P1, _, _ = _fluid_momentum(o, c)
        row = o.series()[-1, 0]
        F = row[0:3] + row[6:9]
        err = max(err, np.abs((P1 - P0) + F + o.edge_me()[:3]).max())
        scale = max(scale, np.abs(F).max())
        n_imp += int(np.abs(row[6:9]).max() > 0)
        P0 = P1
    assert n_imp > 10  # rotation alone covers and uncovers nodes
    assert err <= 1e-12 * scale
