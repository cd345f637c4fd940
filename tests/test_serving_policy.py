"""Queue order of the serving loops (host logic, no GPU)."""
import pytest

from paper_1407_4524_gb300 import serving


def _req(n, steps):
    return dict(lattice="D2Q9", n=n, tau=0.8, steps=steps)


def test_fifo_takes_the_head():
    q = [_req((64, 64), 5000), _req((8, 8), 10)]
    assert serving._next_index(q, "fifo") == 0


def test_sjf_takes_the_smallest_work_first_ties_in_arrival_order():
    q = [_req((64, 64), 5000), _req((32, 32), 100), _req((16, 16), 400), _req((32, 32), 100)]
    assert serving._next_index(q, "sjf") == 1  # 32*32*100 = 16*16*400, arrived first
    q.pop(1)
    assert serving._next_index(q, "sjf") == 1  # 16*16*400 arrived before the other 32x32 request
    assert serving._next_index([q[0]], "sjf") == 0


def test_unknown_policy_is_rejected():
    with pytest.raises(ValueError):
        serving._next_index([_req((8, 8), 1), _req((8, 8), 2)], "lifo")
