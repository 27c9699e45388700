"""GB300-native pseudo-time residual sweep of the variable-density
artificial-compressibility scheme of Leakey, Glenis & Hewett (arXiv 2108.08769).

* ``ac``        -- ctypes binding of the C ABI (include/ac.h); the CUDA
                   library ``libacgb300.so`` does all the numerical work.
* ``workloads`` -- seeded synthetic problems shaped like the paper's tests.
* ``build``     -- in-tree nvcc build for sm_103a.
"""
__all__ = ["ac", "workloads", "build"]
