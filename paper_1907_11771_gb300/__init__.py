"""GB300 (sm_103a) extrapolated-GBS time stepper for method-of-lines wave systems.

Ellison & Fornberg, "A parallel-in-time approach for wave-type PDEs", arXiv 1907.11771.

Modules:
  binding  -- ctypes binding of libgbs.so (the C ABI of include/gbs.h, same names)
  solver   -- GBSSolver, an object wrapper over the binding (torch tensors in, no compute)
  schemes  -- the extrapolation schemes printed in the paper, as data
  inputs   -- seeded synthetic workloads (initial states, media, receivers)
  build    -- nvcc build of libgbs.so for sm_103a
"""
__version__ = "0.1.0"
