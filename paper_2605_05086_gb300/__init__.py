"""GB300-native best-shift tabu search (Sec. 3.1 of "CHAP: A Hybrid GPU-CPU Heuristic for MIP").

Modules:
  instances -- seeded synthetic MIP instances (data only);
  chap      -- ctypes binding of libchap.so, the CUDA library behind include/chap.h;
  build     -- in-tree nvcc build of libchap.so for sm_103a.

Importing the package loads nothing; chap.load() loads the CUDA library and
raises when it is missing.
"""
