"""GB300-native TurboGS sparse-sampled rasterizer path.

The compute lives in ``libturbogs.so`` (hand-written sm_103a CUDA kernels behind
the C ABI declared in ``include/turbogs.h``); ``binding`` exposes those entry
points to Python under the same names.  Importing this package does not load
the library; ``binding`` does, and raises if it is missing.
"""
__all__ = ["binding", "scenes", "config"]
__version__ = "0.1.0"
