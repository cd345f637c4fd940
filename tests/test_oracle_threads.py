"""The oracle's results do not depend on its thread count: OpenMP runs only
over loops whose order does not matter, so one thread and several give the
same bits (the FP64 GPU mode is compared with it bit for bit, and the timed
CPU baseline runs it on every core)."""
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
import numpy as np
sys.path.insert(0, {root!r})
import oracle
cases = [
    dict(lattice="D2Q9", n=(61, 47), tau=0.7, refill="extrap", u0=(0.02, 0.0),
         bodies=[dict(shape="cylinder", R=6.3, X0=(20.4, 23.1), U=(0.03, 0.0), W=0.002),
                 dict(shape="ellipse", R=7.2, R2=3.9, theta0=0.4, X0=(44.2, 22.7), W=0.004)]),
    dict(lattice="D2Q9", n=(50, 70), tau=0.7, gravity=(0.0, -2e-4), edges={{"x": ("wall", "wall")}},
         edge_rule="zouhe",
         bodies=[dict(shape="ellipse", R=9.4, R2=4.7, theta0=0.785398, X0=(25.3, 35.2), free=True,
                      density_ratio=1.5)]),
    dict(lattice="D3Q19", n=(24, 22, 21), tau=0.8, u0=(0.01, 0.0, 0.005), refill="ubar",
         bodies=[dict(shape="sphere", R=4.6, X0=(10.2, 11.3, 9.8), U=(0.02, -0.01, 0.0), W=(0.0, 0.003, 0.001))]),
]
out = {{}}
for k, spec in enumerate(cases):
    o = oracle.Oracle(spec)
    o.step(25)
    out[f"f{{k}}"] = o.f()
    out[f"s{{k}}"] = o.series()
    out[f"b{{k}}"] = o.body_state()
np.savez(sys.argv[1], **out)
"""


def _run(tmp_path, threads):
    path = tmp_path / f"t{threads}.npz"
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT), str(path)], env=env, check=True,
                   timeout=600)
    return np.load(path)


def test_oracle_is_built_with_openmp():
    """The thread-count test below and the CPU baseline's core count mean
    something only if the oracle really runs on several threads."""
    code = f"import sys; sys.path.insert(0, {ROOT!r}); import oracle; print(oracle.threads())"
    env = dict(os.environ, OMP_NUM_THREADS="3")
    out = subprocess.run([sys.executable, "-c", code], env=env, check=True, capture_output=True, text=True,
                         timeout=300)
    assert int(out.stdout.strip().splitlines()[-1]) == 3


def test_oracle_is_independent_of_thread_count(tmp_path, oracle_mod):
    a = _run(tmp_path, 1)
    b = _run(tmp_path, 3)
    assert sorted(a.files) == sorted(b.files)
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k
