"""GB300-native (sm_103a) engine for the time-dependent MPS simulation of
quantum circuits (SaiToh 2011, Sec. 3): the per-gate Vidal update
theta -> SVD -> truncation -> rewrite, behind the C ABI of include/mps.h.

``paper_1111_3124_gb300.mps`` is the ctypes binding of that ABI;
``paper_1111_3124_gb300.circuits`` generates seeded synthetic inputs.
"""

__all__ = ["mps", "circuits", "build"]
