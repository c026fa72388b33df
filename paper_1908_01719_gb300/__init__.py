"""GB300-native finite-element Bloch-Torrey solver for diffusion MRI.

The compute path lives in ``libbtgpu.so`` (CUDA for sm_103a behind the C ABI
of include/bt.h); ``bt`` is its thin ctypes binding and ``simulate`` a
convenience driver that only marshals arguments.
"""
from . import bt  # noqa: F401
from .simulate import Simulation, simulate  # noqa: F401
