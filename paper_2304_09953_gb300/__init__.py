"""GB300-native ligand docking and scoring (paper arXiv:2304.09953, LIGATE).

The compute path is libligate.so (hand-written sm_103a CUDA kernels behind
the C ABI of include/ligate.h); ``native`` is its thin ctypes binding and
``docking`` a small convenience layer over it.  ``workload`` draws seeded
synthetic inputs.  PyTorch is only used by callers for device memory and
streams.
"""
from . import build, native  # noqa: F401

__all__ = ["build", "native", "docking", "workload"]
