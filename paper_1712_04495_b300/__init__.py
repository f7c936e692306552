"""Memory-safe GPU co-scheduling on one B300 (arXiv 1712.04495, schedGPU).

The C ABI lives in ``libschedgpu.so`` (``include/schedgpu.h``); ``abi``
binds it with the same names. ``runtime`` adds torch plumbing (device pool,
streams, device copies of job traces) around those calls. ``tracegen``
builds the seeded synthetic traces.
"""
import os as _os

# Stream slots run jobs concurrently only if they map to distinct hardware
# work queues; the default of 8 would serialise unrelated jobs. Must be set
# before the CUDA context exists.
_os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from . import tracegen  # noqa: E402,F401

__all__ = ["abi", "runtime", "tracegen", "build"]
