"""Pins of the oracle's Zou-He edge rule (walls and inlet as on-node
velocity conditions; the edge treatment of the paper's test section).

  * Poiseuille: a body-force-driven channel between Zou-He walls at the node
    rows 0 and ny - 1 reaches u(y) = g y (H - y) / (2 nu rho0), H = ny - 1,
    to round-off (the condition is exact for the parabola) -- a wrong
    coefficient, sign or tangential term, or a missing force shift, breaks it;
  * the closure: after any step the wall nodes carry u = 0 and the inlet
    nodes the prescribed velocity (uniform and on-node parabola), both
    lattices, both equilibria, random states;
  * a uniform stream through a Zou-He inlet and the zero-gradient outlet is a
    fixed point; fluid at rest in a closed Zou-He box (edges and corners
    included) stays at rest;
  * corner nodes: zero momentum and the density of the inner diagonal
    neighbour.
"""
import numpy as np
import pytest


def _macro(o):
    m = o.macro()  # [4, nz, ny, nx]: rho, ux, uy, uz
    return m


@pytest.mark.parametrize("eq", ["incomp", "standard"])
@pytest.mark.parametrize("tau", [0.55, 0.8, 1.4])
def test_poiseuille_exact_between_zouhe_walls(oracle_mod, tau, eq):
    ny, g = 17, 1e-6
    o = oracle_mod.Oracle(dict(lattice="D2Q9", n=(1, ny), tau=tau, eq=eq, force=(g, 0.0),
                               edges={"x": "periodic", "y": ("wall", "wall")}, edge_rule="zouhe"))
    nu = (tau - 0.5) / 3.0
    o.step(int(12 * (ny - 1) ** 2 / nu))
    ux = _macro(o)[1, 0, :, 0]
    H, y = ny - 1, np.arange(ny)
    exact = g * y * (H - y) / (2.0 * nu)
    assert np.abs(ux - exact).max() <= 1e-9 * exact.max()
    assert abs(ux[0]) <= 1e-15 and abs(ux[-1]) <= 1e-15


def test_poiseuille_exact_d3q19(oracle_mod):
    ny, g, tau = 13, 1e-6, 0.7
    o = oracle_mod.Oracle(dict(lattice="D3Q19", n=(2, ny, 2), tau=tau, force=(0.0, 0.0, g),
                               edges={"x": "periodic", "y": ("wall", "wall"), "z": "periodic"},
                               edge_rule="zouhe"))
    nu = (tau - 0.5) / 3.0
    o.step(int(12 * (ny - 1) ** 2 / nu))
    uz = _macro(o)[3, 0, :, 0]
    H, y = ny - 1, np.arange(ny)
    exact = g * y * (H - y) / (2.0 * nu)
    assert np.abs(uz - exact).max() <= 1e-9 * exact.max()


def _random_state(o, rng, amp=0.01):
    f = o.f()
    o.set_f(f * (1.0 + amp * rng.standard_normal(f.shape)))


@pytest.mark.parametrize("eq", ["incomp", "standard"])
@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
@pytest.mark.parametrize("profile", ["uniform", "parabolic"])
def test_closure_sets_wall_and_inlet_velocity(oracle_mod, lat, eq, profile):
    U = 0.04
    if lat == "D2Q9":
        spec = dict(lattice=lat, n=(23, 15), tau=0.7, eq=eq, u0=(0.02, 0.0),
                    edges={"x": ("inlet", "outlet"), "y": ("wall", "wall")})
    else:
        spec = dict(lattice=lat, n=(12, 11, 9), tau=0.7, eq=eq, u0=(0.02, 0.0, 0.0),
                    edges={"x": ("inlet", "outlet"), "y": ("wall", "wall"), "z": ("wall", "wall")})
    spec.update(inlet=dict(profile=profile, u=U), edge_rule="zouhe", force=(1e-5, 2e-6) + ((3e-6,) if lat == "D3Q19" else ()))
    o = oracle_mod.Oracle(spec)
    rng = np.random.default_rng(11)
    _random_state(o, rng)
    c, w, opp = oracle_mod.lattice_tables(o.q)
    c = np.asarray(c, float)
    g = np.array(spec["force"] + ((0.0,) if lat == "D2Q9" else ()), float)
    nx, ny, nz = o.shape
    rho0 = 1.0
    for _ in range(3):
        o.step(1)
        f = o.f()  # f(t): the closed populations before collision
        rho = f.sum(0)
        j = np.einsum("qa,qzyx->azyx", c, f) + 0.5 * g[:, None, None, None]
        den = rho0 if eq == "incomp" else rho
        u = j / den
        nfaces = np.zeros((nz, ny, nx), int)  # Zou-He faces a node lies on
        nfaces[:, [0, ny - 1], :] += 1
        nfaces[:, :, 0] += 1
        if lat == "D3Q19":
            nfaces[[0, nz - 1], :, :] += 1
        wall_y = np.zeros((nz, ny, nx), bool)
        wall_y[:, [0, ny - 1], :] = True
        if lat == "D3Q19":
            wall_y[[0, nz - 1], :, :] = True
        face = wall_y & (nfaces == 1)
        assert np.abs(u[:, face]).max() <= 1e-16
        # edges and corners: bounce-back, sum_i c_i f_i = 0 (no force shift there)
        jb = np.einsum("qa,qzyx->azyx", c, f)
        assert np.abs(jb[:, nfaces >= 2]).max() <= 1e-16
        inner = ~wall_y[:, :, 0]
        H = ny - 1
        yy = np.broadcast_to(np.arange(ny)[None, :], (nz, ny))
        want = U if profile == "uniform" else 4.0 * U * yy * (H - yy) / H ** 2
        want = np.broadcast_to(want, (nz, ny))
        assert np.abs(u[0, :, :, 0][inner] - want[inner]).max() <= 1e-16
        assert np.abs(u[1:, :, :, 0][:, inner]).max() <= 1e-16


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_uniform_stream_through_zouhe_inlet_is_fixed_point(oracle_mod, lat):
    U = 0.05
    if lat == "D2Q9":
        spec = dict(lattice=lat, n=(20, 8), tau=0.7, u0=(U, 0.0),
                    edges={"x": ("inlet", "outlet"), "y": "periodic"}, inlet=dict(u=U), edge_rule="zouhe")
    else:
        spec = dict(lattice=lat, n=(12, 6, 5), tau=0.7, u0=(U, 0.0, 0.0),
                    edges={"x": ("inlet", "outlet"), "y": "periodic", "z": "periodic"},
                    inlet=dict(u=U), edge_rule="zouhe")
    o = oracle_mod.Oracle(spec)
    f0 = o.f().copy()
    o.step(20)
    assert np.abs(o.f() - f0).max() <= 1e-15


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_closed_zouhe_box_at_rest_stays_at_rest(oracle_mod, lat):
    if lat == "D2Q9":
        spec = dict(lattice=lat, n=(9, 7), tau=0.8, edges={"x": ("wall", "wall"), "y": ("wall", "wall")})
    else:
        spec = dict(lattice=lat, n=(6, 5, 7), tau=0.8,
                    edges={"x": ("wall", "wall"), "y": ("wall", "wall"), "z": ("wall", "wall")})
    o = oracle_mod.Oracle(dict(spec, edge_rule="zouhe"))
    f0 = o.f().copy()
    o.step(10)
    assert np.abs(o.f() - f0).max() <= 1e-15  # a few rounding steps


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_corner_nodes_take_inner_density_and_zero_momentum(oracle_mod, lat):
    if lat == "D2Q9":
        spec = dict(lattice=lat, n=(9, 8), tau=0.8, edges={"x": ("wall", "wall"), "y": ("wall", "wall")})
        corners = [(0, 0, 0, (1, 1, 0)), (8, 7, 0, (7, 6, 0)), (0, 7, 0, (1, 6, 0))]
    else:
        spec = dict(lattice=lat, n=(6, 7, 8), tau=0.8,
                    edges={"x": ("wall", "wall"), "y": ("wall", "wall"), "z": ("wall", "wall")})
        corners = [(0, 0, 0, (1, 1, 1)), (5, 6, 7, (4, 5, 6)), (0, 3, 0, (1, 3, 1)), (2, 6, 7, (2, 5, 6))]
    o = oracle_mod.Oracle(dict(spec, edge_rule="zouhe"))
    rng = np.random.default_rng(5)
    _random_state(o, rng, 0.02)
    c, _, _ = oracle_mod.lattice_tables(o.q)
    c = np.asarray(c, float)
    for _ in range(2):
        fh = o.fhat()
        o.step(1)
        f = o.f()
        for x, y, z, (xi, yi, zi) in corners:
            assert f[:, z, y, x].sum() == pytest.approx(fh[:, zi, yi, xi].sum(), abs=1e-15)
            assert np.abs(c.T @ f[:, z, y, x]).max() <= 1e-16
