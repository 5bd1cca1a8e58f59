"""GB300-native state-vector engine for the quantum-computer simulator of
arXiv:1805.04708 (JUQCS): hand-written sm_103a CUDA kernels behind a C ABI
(``include/qsim.h``), with a thin ctypes binding in ``qsim``.

Import ``paper_1805_04708_gb300.qsim`` for the binding (it loads the compiled
library and raises if it is missing); ``workloads`` holds the seeded input
generators and imports nothing compiled.
"""
__all__ = ["qsim", "workloads"]
