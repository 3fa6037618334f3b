"""GB300-native encrypted 1:N iris matching (CCMM + fold hot path of arxiv 2601.17561).

Submodules: `icm` (ctypes binding of libicm.so, same names as include/icm.h), `engine`
(PyTorch-allocated buffers around the C ABI), `build` (nvcc build of the library for sm_103a),
`synth` (seeded synthetic iris templates).
"""
__all__ = ["icm", "engine", "build", "synth"]
