"""Pins of the oracle's lattice tables and equilibrium (CPU only).

The paper uses D2Q9 (Sec. 4) and names directions only by index (Sec. 3,
Fig. 2: i=1 axis-parallel, i=5 diagonal); D3Q19 is the standard 3-D set.
The quadrature conditions below are what Sec. 2 requires of c_i and w_i:
moments of order 0, 1 and 2 exact (and the 4th-order isotropy that makes the
truncated Maxwellian reproduce Navier-Stokes).
"""
import itertools

import numpy as np
import pytest


@pytest.mark.parametrize("q", [9, 19])
def test_quadrature_conditions(oracle_mod, q):
    c, w, opp = oracle_mod.lattice_tables(q)
    D = 2 if q == 9 else 3
    c = c[:, :D].astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w @ c, 0.0, atol=1e-16)
    M2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(M2, np.eye(D) / 3.0, atol=1e-16)
    # odd moments vanish
    M3 = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.allclose(M3, 0.0, atol=1e-16)
    # 4th-order isotropy: (d_ab d_cd + d_ac d_bd + d_ad d_bc) / 9
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    I = np.eye(D)
    iso = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
           + np.einsum("ad,bc->abcd", I, I)) / 9.0
    assert np.allclose(M4, iso, atol=1e-16)


@pytest.mark.parametrize("q", [9, 19])
def test_opposites_and_ordering(oracle_mod, q):
    c, w, opp = oracle_mod.lattice_tables(q)
    assert (c[0] == 0).all()
    for i in range(q):
        assert opp[opp[i]] == i
        assert (c[opp[i]] == -c[i]).all()
        assert w[opp[i]] == w[i]
    # all velocities distinct, speeds 0, 1, sqrt(2) only
    assert len({tuple(v) for v in c}) == q
    assert set((c * c).sum(1).tolist()) == {0, 1, 2}
    if q == 9:  # Sec. 3 / Fig. 2: i = 1 axis-parallel, i = 5 diagonal
        assert (np.abs(c[1]).sum(), np.abs(c[5]).sum()) == (1, 2)
        assert (c[:, 2] == 0).all()


def _eq_state(oracle_mod, q, eq, rho0=1.0, seed=0):
    """With tau = 1 the oracle's collision returns f^eq(rho, u) of the state."""
    rng = np.random.default_rng(seed)
    n = (4, 3, 1) if q == 9 else (3, 3, 2)
    o = oracle_mod.Oracle(dict(lattice="D2Q9" if q == 9 else "D3Q19", n=n[: 2 if q == 9 else 3],
                               tau=1.0, eq=eq, rho0=rho0))
    c, w, _ = oracle_mod.lattice_tables(q)
    N = n[0] * n[1] * n[2]
    f = w[:, None] * (1.0 + 0.2 * rng.standard_normal((q, N)))
    o.set_f(f)
    return o, f, c.astype(float), w


@pytest.mark.parametrize("q", [9, 19])
@pytest.mark.parametrize("eq", ["incomp", "standard"])
def test_equilibrium_moments(oracle_mod, q, eq):
    """f^eq has the moments that define it: rho, rho0 u (or rho u) and the
    momentum flux rho/3 I + rho0 u u (or rho u u)."""
    rho0 = 1.0 if eq == "standard" else 0.97
    o, f, c, w = _eq_state(oracle_mod, q, eq, rho0=rho0)
    feq = o.fhat().reshape(q, -1)
    rho = f.sum(0)
    j = c.T @ f
    u = j / (rho0 if eq == "incomp" else rho)
    assert np.allclose(feq.sum(0), rho, rtol=0, atol=1e-14)
    assert np.allclose(c.T @ feq, j, rtol=0, atol=1e-14)
    D = 2 if q == 9 else 3
    Pi = np.einsum("ia,ib,in->abn", c, c, feq)[:D, :D]
    rr = rho0 if eq == "incomp" else rho
    want = rho[None, None] / 3.0 * np.eye(D)[:, :, None] + rr * np.einsum("an,bn->abn", u[:D], u[:D])
    assert np.allclose(Pi, want, rtol=0, atol=1e-14)
    # third moment: rho0/3 (u_a d_bc + u_b d_ac + u_c d_ab) off the lattice-
    # artifact diagonal a=b=c
    M3 = np.einsum("ia,ib,ic,in->abcn", c, c, c, feq)[:D, :D, :D]
    I = np.eye(D)
    uu = (u[:D] * (rho0 if eq == "incomp" else rho))
    want3 = (np.einsum("an,bc->abcn", uu, I) + np.einsum("bn,ac->abcn", uu, I)
             + np.einsum("cn,ab->abcn", uu, I)) / 3.0
    for a, b, cc in itertools.product(range(D), repeat=3):
        if a == b == cc:
            continue
        assert np.allclose(M3[a, b, cc], want3[a, b, cc], atol=1e-14)
