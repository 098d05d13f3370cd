"""GB300-native CTMRG for a 2x2 iTPS unit cell (TeNeS, arXiv:2112.13184, Sec. 2.2).

The compute path is libctm.so (CUDA, sm_103a) behind the C ABI in
include/ctm.h; ``paper_2112_13184_gb300.ctm`` is its ctypes binding.
Build the library with ``paper_2112_13184_gb300.build.build()``.
"""
