"""B300-native point-cloud ray launcher (arXiv 2402.13747): voxelisation, coarse
path tracing and exact-path refinement as CUDA kernels behind the C ABI in
include/nimbus.h.

Submodules: ``config`` (method parameters), ``scenes`` (seeded synthetic inputs),
``build`` (nvcc build of libnimbus.so), ``_abi`` (ctypes binding), ``serve``
(continuous-batching request loop).
"""
__all__ = ["config", "scenes"]
