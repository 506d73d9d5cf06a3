"""GB300-native engine for exact mesh-mesh min/max distance (gDist's hot path).

  gdist   -- ctypes binding of the C ABI in include/gdist.h (libgdist.so)
  synth   -- seeded synthetic meshes and rigid transforms
  build   -- nvcc build of libgdist.so for sm_103a

The binding is loaded on first use and raises if the CUDA library is missing;
nothing here computes distances on the CPU.
"""

from . import synth  # noqa: F401

__all__ = ["synth", "gdist", "build"]
