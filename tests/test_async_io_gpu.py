"""Reads that wait only for the steps they need, and body updates that do not
synchronise: the pipelined use (enqueue step t+1, then read the row of step
t; update the kinematics before every step) gives exactly the results of the
synchronous use."""
import numpy as np
import pytest

from test_parity_gpu import CASES_2D, CASES_3D

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,name", [("2d", "moving_cylinders_periodic"), ("3d", "moving_spheres_periodic")])
def test_pipelined_reads_and_updates_match_synchronous(dim, name, prec):
    from paper_1407_4524_gb300 import lbm
    spec = dict((CASES_2D if dim == "2d" else CASES_3D)[name], precision=prec)
    steps = 40 if dim == "2d" else 15
    ref = lbm.Domain(spec, device=0)
    ref.step(steps)
    want = ref.force_torque("lattice")
    ref.close()

    dom = lbm.Domain(spec, device=0)
    nb = len(dom.bodies)
    row = np.zeros((1, nb, 6))
    got = np.zeros((steps, nb, 6))
    for k in range(steps):
        dom.update_bodies(list(dom.bodies))  # same kinematics, uploaded without a host sync
        dom.step(1)
        if k >= 1:  # the previous step's row while this step may still run
            assert dom.lib.lbm_get_force_torque(dom.h, k - 1, 1, 1, row.ctypes.data) == 0
            got[k - 1] = row[0]
    assert dom.lib.lbm_get_force_torque(dom.h, steps - 1, 1, 1, row.ctypes.data) == 0
    got[steps - 1] = row[0]
    assert np.array_equal(got, want)
    assert np.array_equal(dom.force_torque("lattice"), want)
    dom.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("dim,name", [("2d", "moving_cylinders_periodic"), ("2d", "zouhe_box_rotating"),
                                      ("3d", "moving_spheres_periodic"), ("3d", "channel_sphere")])
def test_graph_replay_matches_step_by_step(dim, name, prec):
    """lbm_step(n) replays captured 16-step graphs (the kernels read their step
    index on the device); one-step calls launch kernel by kernel: the results
    are bit-identical, with and without kernel timing."""
    from paper_1407_4524_gb300 import lbm
    spec = dict((CASES_2D if dim == "2d" else CASES_3D)[name], precision=prec)
    steps = 37  # a graph replay, a plain step to even parity, another replay, plain remainder
    ref = lbm.Domain(spec, device=0)
    for _ in range(steps):
        ref.step(1)
    want_ft = ref.force_torque("lattice") if ref.bodies else None
    want_f = ref.populations()
    ref.close()
    for timing in (False, True):
        dom = lbm.Domain(spec, device=0)
        dom.set_kernel_timing(timing)
        dom.step(1)
        dom.step(steps - 1)
        if timing:
            n, ms = dom.kernel_time()
            assert n > 0 and ms > 0.0
        if want_ft is not None:
            assert np.array_equal(dom.force_torque("lattice"), want_ft)
        assert np.array_equal(dom.populations(), want_f)
        assert dom.t == steps
        dom.close()


def test_free_body_graph_replay_matches():
    from paper_1407_4524_gb300 import lbm
    from test_free_gpu import CASES as FREE
    name = sorted(FREE)[0]
    spec = dict(FREE[name], precision="fp32")
    ref = lbm.Domain(spec, device=0)
    for _ in range(40):
        ref.step(1)
    want = ref.body_state()
    ref.close()
    dom = lbm.Domain(spec, device=0)
    dom.step(40)
    assert np.array_equal(dom.body_state(), want)
    dom.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_prepared_graph_matches_step_by_step(prec):
    """lbm_prepare_graph records the 16-step graph at an odd step without
    stepping; the runs that replay it afterwards give the bits of one-step
    calls, and it refuses before the first step of a body set."""
    from paper_1407_4524_gb300 import lbm
    spec = dict(CASES_3D["moving_spheres_periodic"], precision=prec)
    steps = 40
    ref = lbm.Domain(spec, device=0)
    for _ in range(steps):
        ref.step(1)
    want_ft = ref.force_torque("lattice")
    want_f = ref.populations()
    ref.close()
    dom = lbm.Domain(spec, device=0)
    with pytest.raises(lbm.LbmError, match="LBM_ERR_STATE"):
        dom.prepare_graph()
    dom.step(3)  # odd step
    dom.prepare_graph()
    dom.prepare_graph()  # already recorded: nothing to do
    assert dom.t == 3
    dom.step(steps - 3)  # one plain step, two replays, plain remainder
    assert dom.t == steps
    assert np.array_equal(dom.force_torque("lattice"), want_ft)
    assert np.array_equal(dom.populations(), want_f)
    dom.close()
