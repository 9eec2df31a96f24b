"""GB300-native (sm_103a) GeoSSTV P-PDS solver (Takemoto & Ono, arXiv 2510.00562).

Modules:
  binding  -- ctypes binding of the C ABI in include/gsstv.h (libgsstv.so)
  solver   -- torch-facing wrapper (device memory and streams only)
  build    -- in-tree nvcc build of libgsstv.so for sm_103a
  synth    -- seeded synthetic cubes (inputs only, none of the method)
  metrics  -- MPSNR / MSSIM of Sec. IV-A
Nothing is imported eagerly: the CUDA library is loaded on first use.
"""
__version__ = "0.1.0"
