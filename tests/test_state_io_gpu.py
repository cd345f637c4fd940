"""Setting and reading the state through the C ABI (lbm_set_populations,
lbm_get_macros) against the FP64 oracle, from seeded random states: the
parity cases of test_parity_gpu otherwise all start from an equilibrium."""
import numpy as np
import pytest

from parity_util import TOL_FP16_FT, TOL_FP16_POP, TOL_FP64_POP, TOL_RED_FT, TOL_RED_POP, ft_rel_error, pop_error
from test_parity_gpu import CASES_2D, CASES_3D

pytestmark = pytest.mark.gpu

NAMES = [("2d", "channel_cylinder"), ("2d", "moving_cylinders_periodic"), ("2d", "zouhe_box_rotating"),
         ("2d", "refill_extrap_ellipse"), ("3d", "moving_spheres_periodic"), ("3d", "zouhe_duct_sphere")]


def _random_f(ref, seed, amp=0.01):
    rng = np.random.default_rng(seed)
    f = ref.f()
    return f * (1.0 + amp * rng.standard_normal(f.shape))


def _pair(oracle_mod, spec, seed):
    from paper_1407_4524_gb300 import lbm
    ref = oracle_mod.Oracle(spec)
    f = _random_f(ref, seed)
    ref.set_f(f)
    dom = lbm.Domain(spec, device=0)
    dom.set_populations(f)
    return dom, ref


@pytest.mark.parametrize("dim,name", NAMES)
def test_fp64_from_random_state_bit_identical(oracle_mod, dim, name):
    spec = dict((CASES_2D if dim == "2d" else CASES_3D)[name], precision="fp64")
    dom, ref = _pair(oracle_mod, spec, 17)
    solid = ref.solid()
    assert pop_error(dom.populations(), ref.fhat(), solid) == 0.0  # collided exactly as the oracle
    m_gpu, m_ref = dom.macros(), ref.macro()
    assert np.abs(m_gpu - m_ref).max() <= 1e-14
    steps = 60 if dim == "2d" else 20
    dom.step(steps)
    ref.step(steps)
    assert np.array_equal(dom.solid(), ref.solid())
    assert pop_error(dom.populations(), ref.fhat(), ref.solid()) <= TOL_FP64_POP
    if ref.bodies:
        for kind in ("static", "lattice", "moving"):
            assert np.array_equal(dom.force_torque(kind), ref.force_torque(kind)), kind
    assert np.abs(dom.macros() - ref.macro()).max() <= 1e-14


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("dim,name", NAMES)
def test_reduced_from_random_state(oracle_mod, dim, name, prec):
    spec = dict((CASES_2D if dim == "2d" else CASES_3D)[name], precision=prec)
    dom, ref = _pair(oracle_mod, spec, 29)
    steps = 60 if dim == "2d" else 20
    dom.step(steps)
    ref.step(steps)
    pop_tol = TOL_RED_POP if prec == "fp32" else TOL_FP16_POP
    assert pop_error(dom.populations(), ref.fhat(), ref.solid()) <= pop_tol
    m_gpu, m_ref = dom.macros(), ref.macro()
    assert np.abs(m_gpu - m_ref).max() <= (2e-6 if prec == "fp32" else 2e-4)
    if ref.bodies:
        ft_tol = TOL_RED_FT if prec == "fp32" else TOL_FP16_FT
        for kind in ("static", "lattice", "moving"):
            assert ft_rel_error(dom.force_torque(kind), ref.force_torque(kind), spec=spec) <= ft_tol, kind


def test_set_populations_rejects_null():
    from paper_1407_4524_gb300 import lbm
    dom = lbm.Domain(dict(CASES_2D["no_bodies_ragged"], precision="fp32"), device=0)
    assert dom.lib.lbm_set_populations(dom.h, None) == 1  # LBM_ERR_ARG
    assert dom.lib.lbm_get_macros(dom.h, None) == 1  # LBM_ERR_ARG
