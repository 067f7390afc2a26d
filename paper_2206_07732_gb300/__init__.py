"""GB300 wave-tank step (arxiv 2206.07732): CUDA library libwec + thin ctypes binding.

Modules:
  wec    -- binding of include/wec.h (Tank, Poisson, wave utilities)
  build  -- nvcc build of libwec.so for sm_103a
  synth  -- seeded synthetic workloads (no method arithmetic)
Importing the package loads nothing; ``wec.load()`` loads the library.
"""
