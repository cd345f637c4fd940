"""Serving batch (lbm_batch_*): continuous batching of static-body solves.

A solve's force/torque series must be the same alone in the serving system
(a batch that holds only it) and in any mix: every solve of a batch runs the
same per-node arithmetic and the per-body sums are exact fixed point, so the
comparison is bit for bit.  A served solve also matches the same problem
stepped as a standalone domain (another kernel arrangement) within the
reduced-precision tolerance.
Also: admission against the memory budget, rejected problems, release of a
running solve, a batched solve against the FP64 oracle, and the serving loop
against one-solve-at-a-time.
"""
import numpy as np
import pytest

from parity_util import TOL_FP16_FT, TOL_RED_FT, ft_rel_error

pytestmark = pytest.mark.gpu

KINDS = ("static", "lattice", "moving")


def _mix():
    """small requests of both lattices, both reduced precisions, ragged sizes"""
    return [
        dict(id=0, lattice="D2Q9", n=(131, 67), tau=0.62, edges={"x": ("inlet", "outlet"), "y": ("wall", "wall")},
             inlet={"profile": "parabolic", "u": 0.04}, bodies=[dict(shape="cylinder", R=7.3, X0=(33.1, 30.2))],
             precision="fp16", steps=300),
        dict(id=1, lattice="D3Q19", n=(64, 48, 40), tau=0.7, edges={"x": ("inlet", "outlet")},
             inlet={"profile": "uniform", "u": 0.03}, u0=(0.03, 0.0, 0.0),
             bodies=[dict(shape="sphere", R=6.2, X0=(16.4, 23.1, 19.7))], precision="fp32", steps=170),
        dict(id=2, lattice="D2Q9", n=(90, 40), tau=0.9, u0=(0.02, 0.01),
             bodies=[dict(shape="cylinder", R=5.0, X0=(45.5, 20.2))], precision="fp32", steps=257),
        dict(id=3, lattice="D3Q19", n=(40, 36, 33), tau=0.56, u0=(0.02, 0.01, 0.0),
             bodies=[dict(shape="sphere", R=5.5, X0=(20.0, 18.3, 16.1)),
                     dict(shape="sphere", R=4.0, X0=(6.0, 5.0, 5.0))], precision="fp16", steps=95),
        dict(id=4, lattice="D2Q9", n=(64, 64), tau=0.75, precision="fp16", steps=64),  # no body
    ]


def _alone(spec):
    """the solve alone in the serving system: a batch that holds only it"""
    from paper_1407_4524_gb300 import lbm
    batch = lbm.Batch(1 << 31, max_slots=1, ticks_per_launch=16)
    s = batch.admit(spec)
    assert s is not None
    while s not in batch.poll():
        batch.run(4)
    out = {k: batch.force_torque(s, k) for k in KINDS}
    batch.close()
    return out, None


def test_alone_vs_mix_bitwise():
    from paper_1407_4524_gb300 import lbm
    reqs = _mix()
    batch = lbm.Batch(1 << 31, max_slots=8, ticks_per_launch=16)
    slots = {}
    # staggered admission: two first, the rest after some ticks
    for r in reqs[:2]:
        slots[r["id"]] = batch.admit(r)
    batch.run(3)
    for r in reqs[2:]:
        slots[r["id"]] = batch.admit(r)
    assert all(s is not None for s in slots.values())
    finished = set()
    for _ in range(200):
        batch.run(1)
        finished.update(batch.poll())
        if len(finished) == len(reqs):
            break
    assert finished == set(slots.values())
    for r in reqs:
        s = slots[r["id"]]
        assert batch.time(s) == r["steps"]
        ref, _ = _alone(r)
        for k in KINDS:
            got = batch.force_torque(s, k)
            assert got.shape == ref[k].shape
            assert np.array_equal(got, ref[k]), f"request {r['id']} {k}: batch differs from alone"
    batch.close()


def test_each_solve_alone_in_batch_matches_domain():
    from paper_1407_4524_gb300 import lbm
    for r in (_mix()[1], _mix()[2]):
        batch = lbm.Batch(1 << 30, max_slots=2, ticks_per_launch=7)
        s = batch.admit(r)
        while s not in batch.poll():
            batch.run(5)
        # a standalone domain steps its boundary nodes through the cut-link
        # kernel and the stream-collide pass, a served solve through the
        # boundary-node kernel: the same method in other FP32 operation orders
        dom = lbm.Domain(r, device=0, series_capacity=r["steps"])
        dom.step(r["steps"])
        for k in KINDS:
            e = ft_rel_error(batch.force_torque(s, k), dom.force_torque(k), spec=r)
            assert e <= TOL_RED_FT, (r["id"], k, e)
        dom.close()
        batch.close()


def test_admission_budget():
    from paper_1407_4524_gb300 import lbm
    r = _mix()[0]
    probe = lbm.Batch(1 << 30, max_slots=4)
    need = probe.solve_bytes(r)
    probe.close()
    assert need > r["n"][0] * r["n"][1] * 9 * 2 * 2  # at least the two population copies
    batch = lbm.Batch(need + need // 2, max_slots=4, ticks_per_launch=8)
    s0 = batch.admit(r)
    assert s0 is not None
    assert batch.usage() == (1, need)
    assert batch.admit(r) is None  # over budget: nothing allocated
    assert batch.usage() == (1, need)
    batch.release(s0)
    assert batch.usage() == (0, 0)
    s1 = batch.admit(r)
    assert s1 is not None
    batch.close()
    few = lbm.Batch(1 << 31, max_slots=1)
    assert few.admit(_mix()[4]) is not None
    assert few.admit(_mix()[4]) is None  # no free slot
    few.close()


def test_rejects_fp64_and_moving_bodies():
    from paper_1407_4524_gb300 import lbm
    batch = lbm.Batch(1 << 30, max_slots=2)
    r = dict(_mix()[2])
    r["precision"] = "fp64"
    with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
        batch.admit(r)
    r = dict(_mix()[2])
    r["bodies"] = [dict(shape="cylinder", R=5.0, X0=(45.5, 20.2), U=(0.01, 0.0))]
    with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
        batch.admit(r)
    assert batch.usage() == (0, 0)
    batch.close()


def test_release_running_solve_leaves_others_exact():
    from paper_1407_4524_gb300 import lbm
    reqs = _mix()
    batch = lbm.Batch(1 << 31, max_slots=4, ticks_per_launch=10)
    a = batch.admit(reqs[0])
    b = batch.admit(reqs[2])
    batch.run(4)
    batch.release(b)  # still running
    while a not in batch.poll():
        batch.run(4)
    ref, _ = _alone(reqs[0])
    assert np.array_equal(batch.force_torque(a, "static"), ref["static"])
    batch.close()


def test_batched_solve_vs_oracle(oracle_mod):
    from paper_1407_4524_gb300 import lbm
    r = _mix()[2]
    batch = lbm.Batch(1 << 30, max_slots=2, ticks_per_launch=32)
    s = batch.admit(r)
    while s not in batch.poll():
        batch.run(2)
    ref = oracle_mod.Oracle(r)
    ref.step(r["steps"])
    for k in KINDS:
        e = ft_rel_error(batch.force_torque(s, k), ref.force_torque(k), spec=r)
        assert e <= TOL_RED_FT, f"{k}: {e:.3e}"
    batch.close()


def test_serving_loop_matches_sequential():
    from paper_1407_4524_gb300 import serving
    reqs = _mix()
    for k, r in enumerate(reqs):
        r["arrival_s"] = 0.02 * k
    sb, ser_b = serving.serve_batched(reqs, budget_bytes=1 << 31, max_slots=3, ticks_per_launch=16,
                                      keep_series=True)
    ss, ser_s = serving.serve_sequential(reqs, keep_series=True)
    assert sb["requests"] == ss["requests"] == len(reqs)
    # one at a time the solves run as standalone domains (cut-link kernel and
    # stream-collide pass), batched through the boundary-node kernel: the
    # same method in other FP32 operation orders
    for r in reqs:
        a, b = np.asarray(ser_b[r["id"]]), np.asarray(ser_s[r["id"]])
        assert a.shape == b.shape
        if r.get("bodies"):
            tol = TOL_RED_FT if r["precision"] == "fp32" else TOL_FP16_FT
            assert ft_rel_error(a, b, spec=r) <= tol, r["id"]
    assert sb["p50_s"] > 0 and sb["p99_s"] >= sb["p50_s"]


def test_unstable_solve_is_isolated():
    """One solve going unstable is reported for that slot only; the others are
    unaffected (bit-identical to alone)."""
    from paper_1407_4524_gb300 import lbm
    good = _mix()[2]
    bad = dict(lattice="D2Q9", n=(64, 32), tau=0.51, u0=(0.35, 0.0), precision="fp32", steps=40,
               bodies=[dict(shape="cylinder", R=5.0, X0=(32.3, 16.2))])
    batch = lbm.Batch(1 << 30, max_slots=4, ticks_per_launch=16)
    sg, sb = batch.admit(good), batch.admit(bad)
    done = set()
    while len(done) < 2:
        batch.run(2)
        done.update(batch.poll())
    with pytest.raises(lbm.LbmError, match="LBM_ERR_UNSTABLE"):
        batch.force_torque(sb, "static")
    ref, _ = _alone(good)
    assert np.array_equal(batch.force_torque(sg, "static"), ref["static"])
    batch.close()
