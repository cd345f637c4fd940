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
