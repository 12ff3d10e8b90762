"""GB300-native Gaussian ray tracing (GRTX): unit-sphere instance BVH, checkpointed k-buffer
rounds, compositing with early termination, backward pass and a request server, as CUDA
kernels for sm_103a behind a C ABI (libgrtx.so).

Importing the package does not load the native library; `paper_2601_20429_gb300.native`
does, and fails loudly if it has not been built.
"""
__all__ = ["scenes"]
