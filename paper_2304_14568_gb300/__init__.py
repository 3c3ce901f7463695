"""GB300-native ADMM-BB for robust proton treatment planning (sm_103a).

The solver lives in librpt.so (CUDA kernels behind the C ABI of include/rpt.h);
`rpt` is its thin ctypes binding and `build` compiles it in-tree with nvcc.
"""
__all__ = ["rpt", "build"]
