"""GB300-native FFT-accelerated multi-block Poisson solver (Costa, arXiv 2106.03583).

* ``snac``   -- ctypes binding of libsnac.so (the CUDA library; ``include/snac.h`` is its C ABI);
* ``inputs`` -- seeded synthetic problems (block layouts, stretched grids, right-hand sides);
* ``build``  -- compiles libsnac.so in-tree for sm_103a.
"""
__all__ = ["snac", "inputs", "build"]
