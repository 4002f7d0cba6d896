"""GB300-native (sm_103a) cascaded central-moment lattice Boltzmann library.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/lbm.h``); :mod:`paper_1202_6351_gb300.lbm` is its Python binding.
Importing the package loads nothing: the library is loaded on first use.
"""
from . import workloads  # noqa: F401  (seeded inputs; no arithmetic of the method)

__all__ = ["lbm", "workloads", "build"]
