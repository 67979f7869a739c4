"""B300-native NRTO inner loop: CUDA library `libnrto.so` behind a C ABI, with a thin
ctypes binding (`paper_2603_02642_b300.nrto`).  Importing the package does not load the
shared library; `nrto.load()` does, and raises if it is missing."""
