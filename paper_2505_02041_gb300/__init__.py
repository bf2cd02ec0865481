"""GB300-native Holographic Radiance Cascades (HRC) for 2D global illumination.

Layout:
  include/hrc.h (repo root) -- the C ABI
  csrc/                     -- CUDA kernels (sm_103a) and the host runtime
  build.py                  -- nvcc build of libhrc.so
  _lib.py                   -- ctypes binding with the C names
  api.py                    -- HRC context class and torch.autograd wrapper
  scenes.py                 -- seeded synthetic input scenes

Importing the package is cheap; the CUDA library loads on first use.
"""
import importlib

__all__ = ["HRC", "BatchedHRC", "fluence", "fluence_bounces", "build"]


def __getattr__(name):
    if name in ("HRC", "BatchedHRC", "fluence", "fluence_bounces"):
        return getattr(importlib.import_module(__name__ + ".api"), name)
    if name == "build":
        return importlib.import_module(__name__ + ".build").build
    raise AttributeError(name)
