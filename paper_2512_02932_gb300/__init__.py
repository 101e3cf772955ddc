"""Hybrid 2D/3D Gaussian rasterizer for GB300 (sm_103a): the forward and
backward hot path of EGGS (arXiv 2512.02932, Sec. 3.1-3.2, App. C-D) as
hand-written CUDA behind a C ABI (include/hgs.h).

  abi         ctypes binding of libhgs, same entry-point names as the header
  rasterizer  device buffers, Rasterizer, RasterizeFunction (autograd),
              exchange_types
  serving     continuous-batching render loop over resident scenes
  fdo         frequency-decoupled optimisation: Haar DWT image losses and
              the Algorithm 1 backward
  build       nvcc build of libhgs.so
"""
from .abi import HgsError, load  # noqa: F401
from .rasterizer import (RasterizeFunction, Rasterizer, SceneTensors, camera_struct,  # noqa: F401
                         config_struct, exchange_types, rasterize)
