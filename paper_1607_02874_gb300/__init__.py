"""GB300-native reactive lattice Boltzmann step (Falcucci et al. 2016).

The compute path is the CUDA library ``_lib/liblbm.so`` (C ABI declared in
``include/lbm.h``); :mod:`.lbm` is a thin ctypes binding to it. PyTorch only
provides device memory (caching allocator) and streams.
"""
from .lbm import (  # noqa: F401
    BC_PERIODIC,
    BC_PRESSURE,
    BF16_DEV,
    FP16_DEV,
    FP32,
    LAYOUT_AUTO,
    LAYOUT_DENSE,
    LAYOUT_FLUID,
    Geometry,
    LbmError,
    Simulation,
    library,
    request_footprint,
    step_batch,
)
