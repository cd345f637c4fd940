"""Pins of the oracle's curved-wall rule and momentum exchange (CPU only).

What fixes each formula of the paper here:
  * closed-box momentum balance: P_fl(t+1) - P_fl(t) = -F(t) holds exactly
    for Eq. flow_force_2 (static body) and Eq. ForceInMovement (moving body:
    impulsive terms over A+ / A-), and the angular analogue for
    Eqs. flow_torque_2 / TorqueInMovement -- this is the discrete
    Reynolds-transport argument of Sec. 3 and catches any wrong sign, index or
    dropped term in the link sums, the A+/A- sets or the reference point;
  * Galilean invariance: a uniform flow co-moving with a translating body is
    a fixed point of the curved-wall rule (pins the sign of its moving-wall
    term) and gives zero moving-frame force (Eq. ForceInMovementMovingFrame);
  * Delta = 1/2, u_B = 0 reduces the rule to bounce-back (mass conserved);
  * fluid at rest gives F = T = 0; symmetry zeros;
  * Taylor-Couette flow between curved walls converges to the analytic
    profile (both chi branches of Sec. 2.1, moving wall);
  * link geometry against brute force and bisection.
"""
import numpy as np
import pytest


def _tables(oracle_mod, o):
    c, w, opp = oracle_mod.lattice_tables(o.q)
    return c.astype(float), w, opp


def _fluid_momentum(o, c, origin=None):
    """P = sum_fluid sum_i c_i f_i, L = sum_fluid x cross sum_i c_i f_i."""
    f = o.f().reshape(o.q, -1)
    fluid = o.solid().reshape(-1) < 0
    j = (c.T @ f)[:, fluid]
    P = j.sum(1)
    nx, ny, nz = o.shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pos = np.stack([xx.reshape(-1), yy.reshape(-1), zz.reshape(-1)]).astype(float)[:, fluid]
    L = np.cross(pos.T, j.T).sum(0)
    return P, L, f[:, fluid].sum()


def _pose(b, t):
    return np.array(b["X0"], float) + t * np.array(b.get("U", (0, 0, 0)), float)


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_fluid_at_rest_gives_zero_force(oracle_mod, lat):
    if lat == "D2Q9":
        spec = dict(lattice=lat, n=(30, 26), tau=0.7,
                    bodies=[dict(shape="cylinder", R=6.37, X0=(12.3, 11.8))])
    else:
        spec = dict(lattice=lat, n=(16, 15, 14), tau=0.7,
                    bodies=[dict(shape="sphere", R=4.61, X0=(7.2, 7.45, 6.9))])
    o = oracle_mod.Oracle(spec)
    f0 = o.f().copy()
    o.step(5)
    fl = o.solid() < 0
    assert np.abs(o.f()[:, fl] - f0[:, fl]).max() <= 1e-15
    ft = o.force_torque("static")
    assert np.abs(ft).max() <= 1e-14
    assert np.array_equal(o.force_torque("moving"), ft)


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_halfway_body_is_bounce_back_and_conserves_mass(oracle_mod, lat):
    rng = np.random.default_rng(5)
    if lat == "D2Q9":
        spec = dict(lattice=lat, n=(28, 24), tau=0.66, u0=(0.03, 0.01),
                    bodies=[dict(shape="cylinder", R=5.5, X0=(13.0, 11.5), halfway=True)])
    else:
        spec = dict(lattice=lat, n=(14, 12, 12), tau=0.66, u0=(0.03, 0.01, -0.02),
                    bodies=[dict(shape="sphere", R=3.7, X0=(6.5, 6.0, 5.5), halfway=True)])
    o = oracle_mod.Oracle(spec)
    c, w, _ = _tables(oracle_mod, o)
    f = o.f() * (1.0 + 0.02 * rng.standard_normal(o.f().shape))
    o.set_f(f)
    _, _, m0 = _fluid_momentum(o, c)
    o.step(25)
    _, _, m1 = _fluid_momentum(o, c)
    assert abs(m1 - m0) <= 2e-14 * m0


@pytest.mark.parametrize("eq", ["incomp", "standard"])
@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_static_body_momentum_balance_periodic(oracle_mod, lat, eq):
    """Eq. flow_force_2: P_fl(t+1) - P_fl(t) = -F(t) in a periodic box."""
    if lat == "D2Q9":
        spec = dict(lattice=lat, n=(40, 30), tau=0.6, eq=eq, u0=(0.04, 0.015),
                    bodies=[dict(shape="cylinder", R=6.3, X0=(17.4, 14.2))])
    else:
        spec = dict(lattice=lat, n=(20, 16, 15), tau=0.6, eq=eq, u0=(0.04, 0.01, -0.012),
                    bodies=[dict(shape="sphere", R=4.4, X0=(8.3, 7.6, 7.1))])
    o = oracle_mod.Oracle(spec)
    c, _, _ = _tables(oracle_mod, o)
    P = [_fluid_momentum(o, c)[0]]
    for _ in range(12):
        o.step(1)
        P.append(_fluid_momentum(o, c)[0])
    dP = np.diff(np.array(P), axis=0)
    F = o.force_torque("static")[:, 0, :3]
    scale = np.abs(F).max()
    assert scale > 1e-3
    assert np.abs(dP + F).max() <= 1e-12 * scale
    assert np.abs(o.series()[:, 0, 6:12]).max() == 0.0  # no impulsive terms


def _closed_box(lat, bodies, u0, tau=0.7):
    if lat == "D2Q9":
        n = (34, 30)
        edges = {"x": ("wall", "wall"), "y": ("wall", "wall")}
    else:
        n = (18, 16, 15)
        edges = {"x": ("wall", "wall"), "y": ("wall", "wall"), "z": ("wall", "wall")}
    return dict(lattice=lat, n=n, tau=tau, u0=u0, edges=edges, bodies=bodies)


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_torque_balance_closed_box(oracle_mod, lat):
    """Eq. flow_torque_2 with r = x_A - x_0 at the fluid node: in a walled box
    L_fl(t+1) - L_fl(t) = -(T_b + X x F_b) - T_walls (torques about the
    origin), and the same for the momentum."""
    if lat == "D2Q9":
        b = [dict(shape="cylinder", R=5.7, X0=(15.3, 13.6))]
        u0 = (0.03, -0.02)
    else:
        b = [dict(shape="sphere", R=4.2, X0=(8.6, 7.3, 7.7))]
        u0 = (0.03, -0.02, 0.015)
    o = oracle_mod.Oracle(_closed_box(lat, b, u0))
    c, _, _ = _tables(oracle_mod, o)
    X = np.array(b[0]["X0"] + ((0.0,) if lat == "D2Q9" else ()), float)
    P0, L0, _ = _fluid_momentum(o, c)
    errs_p, errs_l, scale_p, scale_l = [], [], 0.0, 0.0
    for _ in range(10):
        o.step(1)
        P1, L1, _ = _fluid_momentum(o, c)
        row = o.series()[-1, 0]
        F, T = row[0:3], row[3:6]
        edge = o.edge_me()
        T_origin = T + np.cross(X, F)
        errs_p.append(np.abs((P1 - P0) + F + edge[:3]).max())
        errs_l.append(np.abs((L1 - L0) + T_origin + edge[3:]).max())
        scale_p = max(scale_p, np.abs(F).max())
        scale_l = max(scale_l, np.abs(T_origin).max())
        P0, L0 = P1, L1
    assert scale_p > 1e-3 and scale_l > 1e-3
    assert max(errs_p) <= 1e-12 * scale_p
    assert max(errs_l) <= 1e-12 * scale_l


@pytest.mark.parametrize("refill", ["uB", "ubar", "extrap"])
@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_moving_body_momentum_balance(oracle_mod, lat, refill):
    """Eqs. ForceInMovement / TorqueInMovement: with the impulsive terms over
    the covered (A+) and uncovered (A-) nodes the closed-box balance stays
    exact for a translating and rotating body (and fails without them), for
    every refill rule (the impulsive term counts whatever the refill wrote)."""
    if lat == "D2Q9":
        b = [dict(shape="cylinder", R=5.6, X0=(14.2, 13.7), U=(0.09, -0.05), W=0.004)]
        u0 = (0.0, 0.0)
    else:
        b = [dict(shape="sphere", R=4.1, X0=(8.2, 7.6, 7.3), U=(0.08, -0.04, 0.05),
                  W=(0.003, -0.002, 0.004))]
        u0 = (0.0, 0.0, 0.0)
    o = oracle_mod.Oracle(dict(_closed_box(lat, b, u0), refill=refill))
    c, _, _ = _tables(oracle_mod, o)
    P0, L0, _ = _fluid_momentum(o, c)
    err_p, err_l, scale, n_imp, err_static = 0.0, 0.0, 0.0, 0, 0.0
    for t in range(30):
        X = _pose(b[0], t)
        if X.size == 2:
            X = np.append(X, 0.0)
        o.step(1)
        P1, L1, _ = _fluid_momentum(o, c)
        row = o.series()[-1, 0]
        F = row[0:3] + row[6:9]
        T = row[3:6] + row[9:12]
        edge = o.edge_me()
        err_p = max(err_p, np.abs((P1 - P0) + F + edge[:3]).max())
        err_l = max(err_l, np.abs((L1 - L0) + T + np.cross(X, F) + edge[3:]).max())
        err_static = max(err_static, np.abs((P1 - P0) + row[0:3] + edge[:3]).max())
        scale = max(scale, np.abs(F).max())
        n_imp += int(np.abs(row[6:9]).max() > 0)
        P0, L0 = P1, L1
    assert n_imp > 3, "the body should cover/uncover nodes in 30 steps"
    assert err_p <= 1e-12 * scale
    assert err_l <= 1e-11 * scale
    assert err_static > 1e-6 * scale  # the static form alone misses the A+/A- momentum
    if refill == "extrap":
        assert o.extrapolated() > 0


@pytest.mark.parametrize("refill", ["uB", "ubar", "extrap"])
@pytest.mark.parametrize("eq", ["incomp", "standard"])
@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_galilean_comoving_uniform_flow(oracle_mod, lat, eq, refill):
    """A uniform flow co-moving with a translating body stays exactly f^eq(1,U)
    through the curved-wall rule, every refill rule (rho_bar = 1 and u_bar =
    u_B = U there; extrapolation of a uniform field is exact) and A+/A-
    changes; the moving-frame force is zero and the lattice-frame force
    reduces to the impulsive rho0 U (N+ - N-) noise."""
    if lat == "D2Q9":
        U = (0.05, 0.03)
        b = [dict(shape="cylinder", R=6.2, X0=(15.3, 14.6), U=U)]
        n = (36, 32)
    else:
        U = (0.05, 0.03, -0.04)
        b = [dict(shape="sphere", R=4.3, X0=(9.3, 8.6, 8.2), U=U)]
        n = (20, 18, 17)
    o = oracle_mod.Oracle(dict(lattice=lat, n=n, tau=0.62, eq=eq, u0=U, bodies=b, refill=refill))
    f0 = o.f()[:, 0, 0, 0].copy()
    o.step(40)
    fl = o.solid() < 0
    dev = np.abs(o.f()[:, fl] - f0[:, None]).max()
    assert dev <= 2e-16 * 40
    Fm = o.force_torque("moving")
    Fs = o.force_torque("static")
    assert np.abs(Fm[..., :3]).max() <= 1e-13
    assert np.abs(Fs[..., :3]).max() <= 1e-13
    imp = o.force_torque("impulsive")[..., :3]
    assert np.abs(imp).max() > 1e-3  # nodes were covered / uncovered


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_uniform_inlet_outlet_channel_is_fixed_point(oracle_mod, lat):
    """Inlet link (Delta = 1/2, u_B = u_in) and zero-gradient outlet keep a
    uniform stream at f^eq(1, U)."""
    U = 0.04
    if lat == "D2Q9":
        spec = dict(lattice=lat, n=(20, 8), tau=0.7, u0=(U, 0.0),
                    edges={"x": ("inlet", "outlet"), "y": "periodic"}, inlet=dict(u=U))
    else:
        spec = dict(lattice=lat, n=(12, 6, 5), tau=0.7, u0=(U, 0.0, 0.0),
                    edges={"x": ("inlet", "outlet"), "y": "periodic", "z": "periodic"},
                    inlet=dict(u=U))
    o = oracle_mod.Oracle(spec)
    f0 = o.f().copy()
    o.step(20)
    assert np.abs(o.f() - f0).max() <= 1e-15


def test_rotating_cylinder_on_node_has_zero_force(oracle_mod):
    """90-degree lattice symmetry about the centre node makes F = 0."""
    L = 31
    b = [dict(shape="cylinder", R=7.3, X0=(15.0, 15.0), W=0.004)]
    o = oracle_mod.Oracle(dict(lattice="D2Q9", n=(L, L), tau=0.7, bodies=b))
    o.step(30)
    for kind in ("static", "lattice", "moving"):
        ft = o.force_torque(kind)
        assert np.abs(ft[:, 0, 5]).max() > 1e-4
        assert np.abs(ft[:, 0, :3]).max() <= 1e-12 * np.abs(ft[:, 0, 5]).max()


def test_translating_cylinder_on_mirror_axis(oracle_mod):
    ny = 30
    b = [dict(shape="cylinder", R=6.4, X0=(12.3, (ny - 1) / 2), U=(0.06, 0.0))]
    o = oracle_mod.Oracle(dict(lattice="D2Q9", n=(48, ny), tau=0.7, bodies=b))
    o.step(40)
    for kind in ("static", "lattice", "moving"):
        ft = o.force_torque(kind)
        drag = np.abs(ft[:, 0, 0]).max()
        assert drag > 1e-3
        assert np.abs(ft[:, 0, 1]).max() <= 1e-12 * drag
        assert np.abs(ft[:, 0, 5]).max() <= 1e-11 * drag


def test_sphere_on_periodic_cross_section_has_no_side_force(oracle_mod):
    """A sphere centred on a node of a periodic y-z cross-section in uniform
    inflow: F_y = F_z = 0 and T = 0 by mirror symmetry."""
    n = (24, 16, 16)
    spec = dict(lattice="D3Q19", n=n, tau=0.6, edges={"x": ("inlet", "outlet")},
                inlet=dict(u=0.04), bodies=[dict(shape="sphere", R=3.6, X0=(8.0, 8.0, 8.0))])
    o = oracle_mod.Oracle(spec)
    o.step(20)
    ft = o.force_torque("static")[:, 0]
    drag = np.abs(ft[:, 0]).max()
    assert drag > 1e-3
    assert np.abs(ft[:, 1:]).max() <= 1e-12 * drag


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_link_geometry_bruteforce(oracle_mod, lat):
    """Cut links are exactly the (fluid x, i) with x - c_i inside the body;
    Delta matches bisection on |x_F - s c_i - X| = R; N_i = N_ib."""
    if lat == "D2Q9":
        b = dict(shape="cylinder", R=7.77, X0=(3.4, 11.2))  # wraps the periodic seam
        spec = dict(lattice=lat, n=(26, 24), tau=0.7, bodies=[b])
    else:
        b = dict(shape="sphere", R=4.93, X0=(1.2, 7.3, 12.8))
        spec = dict(lattice=lat, n=(14, 15, 16), tau=0.7, bodies=[b])
    o = oracle_mod.Oracle(spec)
    c, _, opp = oracle_mod.lattice_tables(o.q)
    cells, dirs, deltas = o.links(0)
    nx, ny, nz = o.shape
    X = np.array(b["X0"] + ((0.0,) if lat == "D2Q9" else ()), float)
    Ls = np.array([nx, ny, nz], float)
    sph = b["shape"] == "sphere"

    def rel(p):
        d = p - X
        return d - Ls * np.floor(d / Ls + 0.5)

    def ins(p):
        d = rel(p)
        r2 = d[0] ** 2 + d[1] ** 2 + (d[2] ** 2 if sph else 0.0)
        return r2 <= b["R"] ** 2

    want = []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                p = np.array([x, y, z], float)
                if ins(p):
                    continue
                for i in range(1, o.q):
                    s = np.mod(p - c[i], Ls)
                    if ins(s):
                        want.append(((z * ny + y) * nx + x, i))
    assert [tuple(v) for v in zip(cells.tolist(), dirs.tolist())] == want
    for cell_, i, dl in zip(cells, dirs, deltas):
        x, y, z = cell_ % nx, (cell_ // nx) % ny, cell_ // (nx * ny)
        d = rel(np.array([x, y, z], float))
        lo, hi = 0.0, 1.0
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            q_ = d - mid * c[i]
            r2 = q_[0] ** 2 + q_[1] ** 2 + (q_[2] ** 2 if sph else 0.0)
            if r2 > b["R"] ** 2:
                lo = mid
            else:
                hi = mid
        assert abs(dl - 0.5 * (lo + hi)) < 1e-12
        assert 0.0 < dl <= 1.0
    counts = np.bincount(dirs, minlength=o.q)
    assert all(counts[i] == counts[opp[i]] for i in range(o.q))
    assert (deltas < 0.5).any() and (deltas >= 0.5).any()


def _couette(oracle_mod, R1, R2, tau=0.8, tip=0.01, steps=None):
    L = int(2 * R2 + 6)
    Xc = (L / 2 + 0.31, L / 2 + 0.17)
    w = tip / R1
    bodies = [dict(shape="cylinder", R=R1, X0=Xc, W=w),
              dict(shape="cylinder", R=R2, X0=Xc, invert=True)]
    o = oracle_mod.Oracle(dict(lattice="D2Q9", n=(L, L), tau=tau, bodies=bodies))
    nu = (tau - 0.5) / 3
    if steps is None:
        steps = int(3.0 * (R2 - R1) ** 2 / nu) + 200
    o.step(steps)
    m = o.macro()[:, 0]
    fl = o.solid()[0] < 0
    yy, xx = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    dx, dy = xx - Xc[0], yy - Xc[1]
    r = np.hypot(dx, dy)
    ut = (-dy * m[1] + dx * m[2]) / np.where(r > 0, r, 1)
    A = -w * R1**2 / (R2**2 - R1**2)
    B = w * R1**2 * R2**2 / (R2**2 - R1**2)
    exact = A * r + B / np.where(r > 0, r, 1)
    err = np.abs(ut - exact)[fl].max() / tip
    return err, o


@pytest.mark.slow
def test_taylor_couette_converges(oracle_mod):
    """Curved moving and fixed walls with arbitrary Delta (both chi branches):
    the steady azimuthal velocity converges to A r + B / r at second order."""
    e1, o1 = _couette(oracle_mod, 6.0, 12.0)
    e2, _ = _couette(oracle_mod, 12.0, 24.0)
    assert e1 < 0.03
    assert e2 < e1 / 2.5
    assert o1.fallbacks >= 0


@pytest.mark.parametrize("tau,tol", [(0.8, 5e-3), (1.0, 2e-2)])
def test_taylor_couette_torque(oracle_mod, tau, tol):
    """Absolute torque: at steady state the fluid's torque on the rotating
    inner cylinder is -4 pi mu B per unit length (B the 1/r coefficient of the
    azimuthal velocity), and the fixed outer cylinder takes the opposite one.
    The solid set does not change under rotation, so the three torque forms
    apply; the moving-frame form differs only by the wall velocity terms.
    Measured: 0.17 % off at tau = 0.8, 1.5 % at tau = 1.0 (the interpolated
    wall's effective position drifts with the viscosity).  Taking the lever
    arm at the wall point instead of the fluid node would be off by ~8 %."""
    R1, R2 = 6.0, 12.0
    _, o = _couette(oracle_mod, R1, R2, tau=tau)
    w = 0.01 / R1
    mu = (tau - 0.5) / 3
    T = -4 * np.pi * mu * w * R1**2 * R2**2 / (R2**2 - R1**2)
    for kind in ("static", "lattice", "moving"):
        ft = o.force_torque(kind)[-1]
        assert abs(ft[0, 5] / T - 1) < tol, (kind, ft[0, 5] / T)
        assert abs(ft[1, 5] / -T - 1) < tol, (kind, ft[1, 5] / -T)


@pytest.mark.parametrize("axis", [(0.0, 0.0, 1.0), (1.0, 2.0, 2.0)])
def test_rotating_sphere_in_shell_torque(oracle_mod, axis):
    """3-D absolute torque (Eq. flow_torque_2 with its cross product in full):
    a sphere R1 spinning at Omega inside a fixed concentric spherical shell R2
    (the inverted sphere) takes the Stokes torque -8 pi mu Omega R1^3 R2^3 /
    (R2^3 - R1^3), the shell the opposite one; about a lattice axis and about
    a skew axis (no lattice symmetry to hide a transposed component).
    Measured 0.25 % (z) and 0.54 % (skew) off, off-axis parts < 0.3 %."""
    R1, R2, tau = 4.3, 8.6, 0.8
    L = int(2 * R2 + 6)
    Xc = (L / 2 + 0.31, L / 2 + 0.17, L / 2 - 0.23)
    W = 0.01 / R1 * np.array(axis) / np.linalg.norm(axis)
    bodies = [dict(shape="sphere", R=R1, X0=Xc, W=tuple(W)), dict(shape="sphere", R=R2, X0=Xc, invert=True)]
    o = oracle_mod.Oracle(dict(lattice="D3Q19", n=(L, L, L), tau=tau, bodies=bodies))
    mu = (tau - 0.5) / 3
    o.step(int(3.0 * (R2 - R1) ** 2 / mu) + 200)
    T = -8 * np.pi * mu * W * R1**3 * R2**3 / (R2**3 - R1**3)
    TT = T @ T
    for kind in ("static", "lattice", "moving"):
        ft = o.force_torque(kind)[-1]
        assert abs(ft[0, 3:6] @ T / TT - 1) < 1e-2, (kind, ft[0, 3:6] @ T / TT)
        assert abs(-ft[1, 3:6] @ T / TT - 1) < 1e-2, (kind, -ft[1, 3:6] @ T / TT)
        assert np.linalg.norm(np.cross(ft[0, 3:6], T)) / TT < 1e-2
