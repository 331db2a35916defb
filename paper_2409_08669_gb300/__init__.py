"""GB300-native AdR-Gaussian rasterization path (arXiv 2409.08669).

The compute path is libadr.so (hand-written sm_103a CUDA behind the C ABI in
include/adr.h).  Python modules:
    scenes    seeded synthetic scenes, cameras and settings (inputs only)
    build     compiles libadr.so in-tree
    _lib      ctypes binding with the C names
    raster    Rasterizer and image_loss: device-tensor wrappers over the C ABI
    autograd  torch.autograd functions for the rasterizer, L_load and L1 + SSIM
    finetune  the load-balancing fine-tune (total loss of Sec. 4.4)
    serve     Server: the continuous-batching renderer (adr_serve_*)
Importing this package does not load CUDA; the library loads on first use.
"""
__all__ = ["scenes", "build", "raster", "autograd", "finetune", "serve"]
