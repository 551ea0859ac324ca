"""GB300-native GIGAQBX: FMM-accelerated QBX for the 2D Laplace single- and
double-layer potentials (Wala & Kloeckner, 2018).

Every step of the evaluation runs in the CUDA kernels of ``libgigaqbx.so``
(``csrc/``), reached through the C ABI of ``include/gigaqbx.h``.  This module
only marshals arguments: numpy arrays (host) or torch CUDA tensors (device)
are passed as raw pointers, torch's current stream is handed to the library.
There is no CPU fallback: without the compiled library the import of the
binding fails.
"""
from ._lib import (  # noqa: F401
    Batch,
    GQ_D,
    GQ_S,
    GQ_SP,
    GigaQBXError,
    Geometry,
    MLP,
    lib,
    library_path,
    params_default,
    params_resolve,
)

__all__ = ["Batch", "Geometry", "MLP", "GigaQBXError", "params_default", "params_resolve", "lib", "library_path", "GQ_S", "GQ_D", "GQ_SP"]
