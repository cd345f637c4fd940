"""State snapshots: a domain restored from lbm_save_state continues exactly
as the saved one does (checkpoint / resume), in every precision mode, with
moving, free and elliptic bodies and both edge rules."""
import numpy as np
import pytest

from test_free_gpu import CASES as FREE
from test_parity_gpu import CASES_2D, CASES_3D

pytestmark = pytest.mark.gpu

CASES = [("2d", "moving_cylinders_periodic"), ("2d", "zouhe_box_rotating"), ("2d", "refill_extrap"),
         ("3d", "moving_spheres_periodic"), ("3d", "zouhe_duct_sphere")]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("dim,name", CASES)
def test_resume_continues_bit_for_bit(dim, name, prec):
    from paper_1407_4524_gb300 import lbm
    spec = dict((CASES_2D if dim == "2d" else CASES_3D)[name], precision=prec)
    k1, k2 = (21, 37) if dim == "2d" else (9, 19)
    a = lbm.Domain(spec, device=0)
    a.step(k1)
    blob = a.save_state()
    a.step(k2)
    want_f = a.populations()
    want_ft = a.force_torque("lattice") if a.bodies else None
    a.close()
    b = lbm.Domain(spec, device=0)
    b.load_state(blob)
    assert b.t == k1
    b.step(k2)
    assert b.t == k1 + k2
    assert np.array_equal(b.populations(), want_f)
    if want_ft is not None:
        assert np.array_equal(b.force_torque("lattice"), want_ft)  # the ring's first rows came with the snapshot
    b.close()


@pytest.mark.parametrize("scheme", ["explicit", "aidun", "predictor"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_resume_free_bodies(prec, scheme):
    """the backward-set scheme carries the impulsive terms of the last
    displacement from step to step: they travel with the snapshot"""
    from paper_1407_4524_gb300 import lbm
    spec = dict(FREE["ellipse_channel"], precision=prec, free_scheme=scheme)
    a = lbm.Domain(spec, device=0)
    a.step(30)
    blob = a.save_state()
    a.step(50)
    want = a.body_state()
    want_ft = a.force_torque("lattice")
    a.close()
    b = lbm.Domain(spec, device=0)
    b.load_state(blob)
    b.step(50)
    assert np.array_equal(b.body_state(), want)
    assert np.array_equal(b.force_torque("lattice"), want_ft)
    b.close()


def test_snapshot_of_another_domain_is_rejected():
    from paper_1407_4524_gb300 import lbm
    spec = dict(CASES_2D["moving_cylinders_periodic"], precision="fp32")
    a = lbm.Domain(spec, device=0)
    a.step(3)
    blob = a.save_state()
    a.close()
    other = lbm.Domain(dict(spec, n=(spec["n"][0] + 2, spec["n"][1])), device=0)
    with pytest.raises(lbm.LbmError):
        other.load_state(blob)
    with pytest.raises(lbm.LbmError):
        other.load_state(b"not a snapshot" + bytes(64))
    other.close()
