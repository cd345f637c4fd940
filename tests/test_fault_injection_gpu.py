"""Allocation failures injected on the host (an allocator callback that
refuses after k allocations): domain creation and body placement report
LBM_ERR_OOM, give back everything they took, and a domain whose body
placement failed is left as created -- no bodies, usable, and able to take
its bodies on a later call."""
import ctypes as C

import numpy as np
import pytest

from test_parity_gpu import CASES_2D

pytestmark = pytest.mark.gpu


class _FailingAllocator:
    def __init__(self, stream_ptr):
        import torch
        self.live = {}
        self.left = None  # allocations still granted (None: no limit)

        def _alloc(nbytes, ctx):
            if self.left is not None:
                if self.left == 0:
                    return None
                self.left -= 1
            ptr = int(torch.cuda.caching_allocator_alloc(int(nbytes), 0, stream_ptr or None))
            self.live[ptr] = int(nbytes)
            return ptr

        def _free(ptr, ctx):
            if ptr:
                assert self.live.pop(int(ptr), None) is not None, "freed twice or never allocated"
                torch.cuda.caching_allocator_delete(int(ptr))

        from paper_1407_4524_gb300 import lbm
        self.alloc = lbm.ALLOC_FN(_alloc)
        self.free = lbm.FREE_FN(_free)


def _desc(spec, fa, stream_ptr):
    from paper_1407_4524_gb300 import lbm
    d, q, n = lbm.domain_desc(spec, 0)
    d.stream = C.c_void_p(stream_ptr)
    d.alloc, d.free = fa.alloc, fa.free
    return d, q, n


def _populations(lib, h, q, n):
    out = np.empty(q * int(np.prod(n)))
    assert lib.lbm_get_populations(h, out.ctypes.data) == 0
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_allocation_failures(prec):
    import torch
    from paper_1407_4524_gb300 import lbm
    lib = lbm.load()
    stream_ptr = int(torch.cuda.current_stream(0).cuda_stream)
    spec = dict(CASES_2D["moving_cylinders_periodic"], precision=prec)
    bodies = lbm.body_array(spec["bodies"])
    nbodies = len(spec["bodies"])
    fa = _FailingAllocator(stream_ptr)

    # creation: every early refusal is reported and nothing stays allocated
    failures = 0
    for k in range(0, 16):
        fa.left = k
        d, q, n = _desc(spec, fa, stream_ptr)
        h = C.c_void_p()
        rc = lib.lbm_create_domain(C.byref(d), C.byref(h))
        fa.left = None
        if rc == 0:
            assert lib.lbm_destroy_domain(h) == 0
            break
        failures += 1
        assert rc == 2, lbm.ERRORS.get(rc, rc)
        assert not fa.live
    assert rc == 0 and failures >= 4
    assert not fa.live

    # reference results: no bodies, then the bodies placed normally
    fa.left = None
    d, q, n = _desc(spec, fa, stream_ptr)
    h_ref = C.c_void_p()
    assert lib.lbm_create_domain(C.byref(d), C.byref(h_ref)) == 0
    assert lib.lbm_step(h_ref, 7) == 0
    want_plain = _populations(lib, h_ref, q, n)
    assert lib.lbm_destroy_domain(h_ref) == 0
    assert not fa.live
    ref = lbm.Domain(spec, device=0)
    ref.step(20)
    want_ft = ref.force_torque("lattice")
    ref.close()

    # body placement refused after k allocations
    d, q, n = _desc(spec, fa, stream_ptr)
    h = C.c_void_p()
    assert lib.lbm_create_domain(C.byref(d), C.byref(h)) == 0
    base = dict(fa.live)
    failures = 0
    for k in range(0, 60, 3):
        fa.left = k
        rc = lib.lbm_set_bodies(h, bodies, nbodies)
        fa.left = None
        if rc == 0:
            break
        failures += 1
        assert rc == 2, lbm.ERRORS.get(rc, rc)
        assert fa.live.keys() == base.keys()  # the partial body buffers were given back
    assert rc == 0 and failures >= 3
    # after a refusal the domain is as created: it steps like one without bodies
    h2 = C.c_void_p()
    d2, _, _ = _desc(spec, fa, stream_ptr)
    assert lib.lbm_create_domain(C.byref(d2), C.byref(h2)) == 0
    fa.left = 0
    assert lib.lbm_set_bodies(h2, bodies, nbodies) == 2
    fa.left = None
    assert lib.lbm_step(h2, 7) == 0
    assert np.array_equal(_populations(lib, h2, q, n), want_plain)
    assert lib.lbm_destroy_domain(h2) == 0
    # the domain whose placement finally succeeded runs like one placed at once
    assert lib.lbm_step(h, 20) == 0
    got = np.zeros((20, nbodies, 6))
    assert lib.lbm_get_force_torque(h, 0, 20, lbm.FT_KIND["lattice"], got.ctypes.data) == 0
    assert np.array_equal(got, want_ft)
    assert lib.lbm_destroy_domain(h) == 0
    assert not fa.live
