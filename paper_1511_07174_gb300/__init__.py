"""gbla: single-GPU dense LU / Cholesky / triangular solves with mixed-precision
GMRES-based refinement, hand-written CUDA kernels for sm_103a behind a C ABI
(include/gbla.h). The Python layer only marshals arguments (device pointers,
sizes, the current CUDA stream) into that ABI; every step of a solve runs in
the library's kernels. Import of this package is cheap: libgbla.so is loaded
on first use, and loading fails loudly when it has not been built.
"""
