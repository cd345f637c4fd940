"""Pins of the oracle's bulk BGK step (Eqs. LBE, collision, streaming; CPU).

Closed forms and invariants that fix the collision and streaming operators:
exact mass and momentum conservation in a periodic box, uniform flow as a
fixed point, the viscous decay rate nu = (tau - 1/2)/3 of a shear wave, the
momentum input of the body force, and the steady Poiseuille profile between
two halfway walls.
"""
import numpy as np
import pytest


def _moments(f, c):
    q = f.shape[0]
    ff = f.reshape(q, -1)
    return ff.sum(), (c.T.astype(float) @ ff).sum(1)


@pytest.mark.parametrize("lat,n", [("D2Q9", (24, 17)), ("D3Q19", (9, 8, 7))])
@pytest.mark.parametrize("eq", ["incomp", "standard"])
def test_periodic_box_conserves_mass_and_momentum(oracle_mod, lat, n, eq):
    rng = np.random.default_rng(3)
    o = oracle_mod.Oracle(dict(lattice=lat, n=n, tau=0.62, eq=eq))
    c, w, _ = oracle_mod.lattice_tables(o.q)
    f0 = w[:, None] * (1.0 + 0.05 * rng.standard_normal((o.q, o.N)))
    o.set_f(f0)
    m0, p0 = _moments(o.f(), c)
    o.step(20)
    m1, p1 = _moments(o.f(), c)
    assert abs(m1 - m0) <= 1e-13 * m0
    assert np.abs(p1 - p0).max() <= 1e-13 * m0


@pytest.mark.parametrize("lat,n", [("D2Q9", (12, 10)), ("D3Q19", (6, 5, 4))])
@pytest.mark.parametrize("eq", ["incomp", "standard"])
def test_uniform_flow_is_fixed_point(oracle_mod, lat, n, eq):
    U = (0.03, -0.02, 0.01) if lat == "D3Q19" else (0.03, -0.02)
    o = oracle_mod.Oracle(dict(lattice=lat, n=n, tau=0.7, eq=eq, u0=U))
    f0 = o.f().copy()
    o.step(15)
    assert np.abs(o.f() - f0).max() <= 1e-16 * 8


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_shear_wave_decay_rate(oracle_mod, lat):
    """u_y(x,t) = A sin(k x) exp(-nu k^2 t) with nu = (tau - 1/2)/3."""
    L, tau, A = 64, 0.8, 1e-4
    n = (L, 2) if lat == "D2Q9" else (L, 2, 2)
    o = oracle_mod.Oracle(dict(lattice=lat, n=n, tau=tau))
    c, w, _ = oracle_mod.lattice_tables(o.q)
    k = 2 * np.pi / L
    nx, ny, nz = o.shape
    x = np.arange(nx)
    uy = np.broadcast_to(A * np.sin(k * x), (nz, ny, nx))
    cu = c[:, 1][:, None, None, None] * uy[None]
    f = w[:, None, None, None] * (1.0 + 3 * cu + 4.5 * cu**2 - 1.5 * uy[None] ** 2)
    o.set_f(f)
    steps = 400

    def amp():
        uyy = o.macro()[2, 0, 0]
        return 2.0 / nx * (uyy * np.sin(k * x)).sum()

    a0 = amp()
    o.step(steps)
    nu_meas = -np.log(amp() / a0) / (k * k * steps)
    nu = (tau - 0.5) / 3.0
    assert abs(nu_meas / nu - 1.0) < 2e-3


def test_body_force_momentum_input(oracle_mod):
    """Guo forcing adds exactly g per node per step in a periodic box."""
    g = (1e-5, -2e-5)
    o = oracle_mod.Oracle(dict(lattice="D2Q9", n=(10, 9), tau=0.9, force=g))
    c, _, _ = oracle_mod.lattice_tables(9)
    _, p0 = _moments(o.f(), c)
    o.step(7)
    _, p1 = _moments(o.f(), c)
    assert np.allclose(p1[:2] - p0[:2], 7 * o.N * np.array(g), rtol=1e-10, atol=0)


def _poiseuille(oracle_mod, tau, ny=64, g=1e-6, steps=None):
    nu = (tau - 0.5) / 3.0
    o = oracle_mod.Oracle(dict(lattice="D2Q9", n=(1, ny), tau=tau,
                               edges={"x": "periodic", "y": ("wall", "wall")}, force=(g, 0.0)))
    if steps is None:
        steps = int(6 * ny * ny / nu)
    o.step(steps)
    return o.macro()[1, 0, :, 0], nu


@pytest.mark.slow
def test_poiseuille_second_difference(oracle_mod):
    """Steady channel flow: u'' = -g/nu at every interior node."""
    g = 1e-6
    u, nu = _poiseuille(oracle_mod, 0.8, g=g)
    d2 = u[2:] - 2 * u[1:-1] + u[:-2]
    assert np.allclose(d2, -g / nu, rtol=1e-6)


@pytest.mark.slow
def test_poiseuille_profile_at_magic_tau(oracle_mod):
    """With halfway walls at y = -1/2 and ny - 1/2 the BGK profile equals the
    analytic parabola when (tau - 1/2)^2 = 3/16 (textbook result, not in the
    paper); at other tau the wall slip is O((tau-1/2)^2)."""
    g, ny = 1e-6, 64
    tau = 0.5 + np.sqrt(3.0) / 4.0
    u, nu = _poiseuille(oracle_mod, tau, ny=ny, g=g)
    y = np.arange(ny)
    exact = g / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.abs(u - exact).max() <= 1e-6 * exact.max()
    # away from the magic value the profile is shifted by a uniform slip
    u2, nu2 = _poiseuille(oracle_mod, 1.2, ny=ny, g=g)
    exact2 = g / (2 * nu2) * (y + 0.5) * (ny - 0.5 - y)
    slip = u2 - exact2
    assert np.ptp(slip) <= 1e-6 * exact2.max()
    assert abs(slip.mean()) > 1e-4 * exact2.max()
