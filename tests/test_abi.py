"""The C-ABI library builds, loads and exports every entry point of
include/lbm.h; its lattice tables equal the oracle's (CPU only, no kernels)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(lbm_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("lbm_create_domain", "lbm_set_bodies", "lbm_step", "lbm_get_force_torque",
                     "lbm_destroy_domain", "lbm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1407_4524_gb300 import lbm
    lib = lbm.load()
    raw = ctypes.CDLL(lbm.library_path())
    missing = [n for n in _declared_functions() if not hasattr(raw, n)]
    assert not missing, missing
    assert lib.lbm_version().decode().startswith("lbm-gb300")


@pytest.mark.parametrize("q", [9, 19])
def test_lattice_tables_match_oracle(oracle_mod, q):
    from paper_1407_4524_gb300 import lbm
    c, w, opp = lbm.lbm_lattice_table(q)
    c2, w2, opp2 = oracle_mod.lattice_tables(q)
    assert np.array_equal(c, c2)
    assert np.array_equal(w, w2)  # bitwise: both are correctly rounded quotients
    assert np.array_equal(opp, opp2)


def test_invalid_descriptor_is_rejected_without_gpu():
    """Argument validation happens before any CUDA call."""
    from paper_1407_4524_gb300 import lbm
    lib = lbm.load()
    d = lbm.lbm_domain_desc()
    d.lattice = 7
    h = ctypes.c_void_p()
    rc = lib.lbm_create_domain(ctypes.byref(d), ctypes.byref(h))
    assert rc == 1 and not h.value
    assert b"lattice" in lib.lbm_last_error()
    d.lattice, d.nx, d.ny, d.nz, d.tau, d.rho0 = 9, 8, 8, 1, 0.4, 1.0
    rc = lib.lbm_create_domain(ctypes.byref(d), ctypes.byref(h))
    assert rc == 1 and b"tau" in lib.lbm_last_error()


def _desc(lbm, spec):
    d, _, _ = lbm.domain_desc(spec, 0)
    return d


def test_batch_solve_bytes_without_gpu():
    """Admission arithmetic is host-only: the bytes a solve would hold."""
    from paper_1407_4524_gb300 import lbm
    from paper_1407_4524_gb300 import workloads as W
    import numpy as np
    lib = lbm.load()
    rng = np.random.default_rng(3)
    r = W.serving_request(rng, lattice="D3Q19", precision="fp16")
    bodies = lbm.body_array(r["bodies"])
    out = ctypes.c_int64()

    def nbytes(spec, steps):
        rc = lib.lbm_batch_solve_bytes(ctypes.byref(_desc(lbm, spec)), bodies, len(spec["bodies"]), steps,
                                       ctypes.byref(out))
        return rc, out.value

    rc, b16 = nbytes(r, 1000)
    assert rc == 0
    n = int(np.prod(r["n"]))
    assert b16 >= 2 * 19 * 2 * n  # two FP16 population copies at least
    rc, b16_long = nbytes(r, 5000)
    assert rc == 0 and b16_long - b16 == 4000 * 18 * 8  # the force/torque series grows with the steps
    rc, b32 = nbytes(dict(r, precision="fp32"), 1000)
    assert rc == 0 and b32 - b16 == 2 * 19 * 2 * n  # FP32 doubles the populations only
    rc, _ = nbytes(dict(r, precision="fp64"), 1000)
    assert rc == 1 and b"LBM_FP32 or LBM_FP16" in lib.lbm_last_error()
    rc, _ = nbytes(r, 0)
    assert rc == 1


def test_batch_rejects_bad_arguments_without_gpu():
    from paper_1407_4524_gb300 import lbm
    lib = lbm.load()
    d = lbm.lbm_batch_desc()
    h = ctypes.c_void_p()
    d.max_slots, d.budget_bytes = 0, 1 << 20
    assert lib.lbm_batch_create(ctypes.byref(d), ctypes.byref(h)) == 1 and not h.value
    d.max_slots, d.budget_bytes = 4, 0
    assert lib.lbm_batch_create(ctypes.byref(d), ctypes.byref(h)) == 1
    d.budget_bytes, d.reserved = 1 << 20, 1
    assert lib.lbm_batch_create(ctypes.byref(d), ctypes.byref(h)) == 1
    slot = ctypes.c_int()
    assert lib.lbm_batch_admit(None, None, None, 0, 10, ctypes.byref(slot)) == 1
    assert lib.lbm_batch_run(None, 1) == 1
    cnt = ctypes.c_int()
    assert lib.lbm_batch_poll(None, None, 0, ctypes.byref(cnt)) == 1
    assert lib.lbm_batch_release(None, 0) == 1
    assert lib.lbm_batch_time(None, 0) == -1
    fn = lib.lbm_get_populations_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert fn(None, None) == 1


def test_edge_rule_validated_without_gpu():
    from paper_1407_4524_gb300 import lbm
    lib = lbm.load()
    h = ctypes.c_void_p()
    spec = dict(lattice="D2Q9", n=(8, 8), tau=0.8, edges={"x": "periodic", "y": ("wall", "wall")})
    d = _desc(lbm, dict(spec, edge_rule="zouhe"))
    d.edge_rule = 5
    assert lib.lbm_create_domain(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"edge rule" in lib.lbm_last_error()
    d = _desc(lbm, dict(spec, n=(8, 2), edge_rule="zouhe"))
    assert lib.lbm_create_domain(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"at least 3 nodes" in lib.lbm_last_error()
    out = ctypes.c_int64()
    d = _desc(lbm, dict(spec, precision="fp32", edge_rule="zouhe"))
    rc = lib.lbm_batch_solve_bytes(ctypes.byref(d), None, 0, 10, ctypes.byref(out))
    assert rc == 1 and b"link edge rule" in lib.lbm_last_error()


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's structures have the header's sizes and field offsets
    (checked by compiling the header with the host C compiler)."""
    import shutil
    import subprocess
    from pathlib import Path
    from paper_1407_4524_gb300 import lbm
    if not shutil.which("gcc"):
        pytest.skip("no host C compiler")
    inc = Path(__file__).resolve().parents[1] / "include"
    structs = {"lbm_domain_desc": lbm.lbm_domain_desc, "lbm_body": lbm.lbm_body, "lbm_stats": lbm.lbm_stats,
               "lbm_batch_desc": lbm.lbm_batch_desc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", str(inc), str(src), "-o", str(exe)], check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                              check=True).stdout.split("\n") if line)
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)


def test_state_bytes_of_null_domain():
    from paper_1407_4524_gb300 import lbm
    lib = lbm.load()
    assert lib.lbm_state_bytes(None) == -1
    assert lib.lbm_save_state(None, None, 0) == 1
    assert lib.lbm_load_state(None, None, 0) == 1
