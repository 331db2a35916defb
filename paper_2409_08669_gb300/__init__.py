"""GB300-native AdR-Gaussian rasterization path (arXiv 2409.08669).

The compute path is libadr.so (hand-written sm_103a CUDA behind the C ABI in
include/adr.h).  Python modules:
    scenes   seeded synthetic scenes, cameras and settings (inputs only)
    build    compiles libadr.so in-tree
    _lib     ctypes binding with the C names
    raster   Rasterizer: device-tensor convenience wrapper over the C ABI
Importing this package does not load CUDA; the library loads on first use.
"""
__all__ = ["scenes", "build", "raster"]
