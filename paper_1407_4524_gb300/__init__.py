"""GB300-native lattice-Boltzmann stream-collide with curved-wall links and
momentum-exchange force/torque (Giovacchini & Ortiz, arXiv:1407.4524).

The compute path is the CUDA library ``liblbm.so`` (C ABI: include/lbm.h);
``lbm`` is its ctypes binding and ``workloads`` builds seeded problem
descriptions.  Importing this package loads nothing heavy; the library is
loaded (and built if missing) on first use.
"""
__all__ = ["lbm", "workloads", "build"]
