"""Memory-safe GPU co-scheduling on one B300 (arXiv 1712.04495, schedGPU).

The C ABI lives in ``libschedgpu.so`` (``include/schedgpu.h``); ``abi``
binds it with the same names. ``runtime`` adds torch plumbing (device pool,
streams, device copies of job traces) around those calls. ``tracegen``
builds the seeded synthetic traces.
"""
from . import tracegen  # noqa: F401

__all__ = ["abi", "runtime", "tracegen", "build"]
