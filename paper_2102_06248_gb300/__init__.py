"""GB300 (sm_103a) charge-conserving, time-integrator-agnostic FEM-PIC.

``fempic`` is the binding of the C ABI declared in ``include/fempic.h``;
``workloads`` generates the seeded synthetic inputs; ``build`` compiles the
CUDA library in-tree.
"""
