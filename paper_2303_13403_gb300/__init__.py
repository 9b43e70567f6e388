"""Gutzwiller-projection PQMC sweep on GB300 (sm_103a).

The compute path is the C-ABI library ``libpqmc.so`` built from ``csrc/``;
``pqmc`` is its thin ctypes binding.  Importing this package does not load
the library; ``paper_2303_13403_gb300.pqmc.load()`` does, and fails loudly
when it has not been built.
"""
from . import workloads  # noqa: F401
