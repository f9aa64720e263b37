"""GB300-native sparse third-order Tucker decomposition (HO-SVD, HOOI, SP, MP).

The compute lives in libtucker.so (CUDA, sm_103a; C ABI in include/tucker.h).  `tucker` is the
Python binding; `synth` draws seeded synthetic inputs; `build` compiles the library."""
__all__ = ["tucker", "synth", "build"]
