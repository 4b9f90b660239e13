"""GB300 (sm_103a) implementation of the enhanced spectral boundary integral
(ESBI) hot path: surface vertical velocity over variable depth and RK4 time
stepping, behind the C ABI of include/sbi.h.

The binding lives in ``paper_2310_19840_gb300.sbi`` (loaded on first use so
that importing the package does not require the built library).
"""

__all__ = ["sbi", "build"]
