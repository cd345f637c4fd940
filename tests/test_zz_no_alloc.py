"""lbm_get_populations_noalloc (fixed device scratch, no allocation) against
lbm_get_populations, called through the C ABI.

Collected last on purpose: it must also pass after every other test has run
in the same process (the scratch is set up once per device).
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 0.0  # same export kernel, same values: the copies must agree exactly


def _noalloc(lib):
    fn = lib.lbm_get_populations_noalloc
    fn.argtypes = [C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    return fn


def _both(dom, fn):
    ref = np.empty(dom.q * dom.N)
    got = np.full(dom.q * dom.N, np.nan)
    assert dom.lib.lbm_get_populations(dom.h, ref.ctypes.data) == 0
    rc = fn(dom.h, got.ctypes.data)
    assert rc == 0, dom.lib.lbm_last_error().decode()
    return ref, got


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_noalloc_matches_populations_two_calls(precision):
    from paper_1407_4524_gb300 import lbm
    spec = dict(lattice="D2Q9", n=(61, 29), tau=0.8, edges={"x": ("inlet", "outlet"), "y": ("wall", "wall")},
                inlet={"profile": "parabolic", "u": 0.05}, bodies=[dict(shape="cylinder", R=6.3, X0=(15.4, 14.2))],
                precision=precision)
    dom = lbm.Domain(spec, device=0)
    fn = _noalloc(dom.lib)
    dom.step(7)
    for _ in range(2):  # two calls in a row reuse the scratch
        ref, got = _both(dom, fn)
        np.testing.assert_allclose(got, ref, rtol=TOL, atol=TOL)
    dom.step(5)  # new state, scratch overwritten
    ref, got = _both(dom, fn)
    np.testing.assert_allclose(got, ref, rtol=TOL, atol=TOL)
    dom.close()


def test_noalloc_d3q19_and_limit():
    from paper_1407_4524_gb300 import lbm
    small = dict(lattice="D3Q19", n=(40, 36, 33), tau=0.6, u0=(0.02, 0.0, 0.01), precision="fp32",
                 bodies=[dict(shape="sphere", R=5.5, X0=(20.0, 18.3, 16.1))])
    dom = lbm.Domain(small, device=0)
    fn = _noalloc(dom.lib)
    dom.step(3)
    for _ in range(2):
        ref, got = _both(dom, fn)
        np.testing.assert_allclose(got, ref, rtol=TOL, atol=TOL)
    dom.close()
    # 128 x 128 x 16 x 19 = 4,980,736 values > 4,194,304: rejected, nothing written
    big = dict(lattice="D3Q19", n=(128, 128, 16), tau=0.6, precision="fp16")
    dom = lbm.Domain(big, device=0)
    out = np.full(dom.q * dom.N, 7.0)
    rc = fn(dom.h, out.ctypes.data)
    assert rc == 1  # LBM_ERR_ARG
    assert "4194304" in dom.lib.lbm_last_error().decode()
    assert np.all(out == 7.0)
    dom.close()


def test_noalloc_with_every_allocation_refused():
    """A caller whose allocator refuses everything (a budget that is full)
    can still export: the refusing allocator makes lbm_get_populations fail
    with LBM_ERR_OOM, while the no-allocation export succeeds, twice in a
    row and after further steps, with the values lbm_get_populations gives
    once allocation is allowed again."""
    import torch
    from paper_1407_4524_gb300 import lbm
    from test_fault_injection_gpu import _FailingAllocator, _desc
    from test_parity_gpu import CASES_2D
    lib = lbm.load()
    fn = _noalloc(lib)
    stream_ptr = int(torch.cuda.current_stream(0).cuda_stream)
    fa = _FailingAllocator(stream_ptr)
    spec = dict(CASES_2D["moving_cylinders_periodic"], precision="fp32")
    d, q, n = _desc(spec, fa, stream_ptr)
    h = C.c_void_p()
    assert lib.lbm_create_domain(C.byref(d), C.byref(h)) == 0
    bodies = lbm.body_array(spec["bodies"])
    assert lib.lbm_set_bodies(h, bodies, len(spec["bodies"])) == 0
    size = q * int(np.prod(n))
    for steps in (5, 9):
        assert lib.lbm_step(h, steps) == 0
        fa.left = 0  # from here on every allocation is refused
        blocked = np.empty(size)
        assert lib.lbm_get_populations(h, blocked.ctypes.data) == 2  # LBM_ERR_OOM
        got = [np.full(size, np.nan), np.full(size, np.nan)]
        for g in got:
            rc = fn(h, g.ctypes.data)
            assert rc == 0, lib.lbm_last_error().decode()
        fa.left = None
        ref = np.empty(size)
        assert lib.lbm_get_populations(h, ref.ctypes.data) == 0
        for g in got:
            np.testing.assert_allclose(g, ref, rtol=TOL, atol=TOL)
    assert lib.lbm_destroy_domain(h) == 0
    assert not fa.live
