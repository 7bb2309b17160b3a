"""FP64 CPU oracle of the charge-conserving FEM-PIC step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The GPU library neither imports it nor links it,
and the two share no source code.
"""
from .oracle import OracleMesh, OracleSim, OracleConfig, build, lib_path  # noqa: F401
