"""FP64 CPU oracle for the LBM step, cut-link wall rule and momentum exchange.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import this
package.  The product library (``paper_1407_4524_gb300``) never imports it,
and this package never imports the product library: both take the same plain
problem description (a dict, see ``paper_1407_4524_gb300.workloads``) and
nothing else.

The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64); this module is the
ctypes marshalling around it.  Citations are to Giovacchini & Ortiz,
arXiv:1407.4524 (section / equation labels of the paper).
"""
from .oracle import Oracle, build, lattice_tables, sincos, threads, SERIES_FIELDS  # noqa: F401
