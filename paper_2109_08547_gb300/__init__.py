"""GB300-native e-ph scattering and coupled electron-phonon BTE (arXiv 2109.08547 hot path).

Modules:
  synthetic  seeded synthetic Wannier models and workloads (inputs only)
  build      nvcc build of the CUDA library (csrc/ -> _build/libephb.so)
  binding    ctypes binding of the C ABI (include/ephb.h)

The binding is imported lazily so that the input generators can be used without the
CUDA library.
"""

__all__ = ["synthetic", "build", "binding"]
