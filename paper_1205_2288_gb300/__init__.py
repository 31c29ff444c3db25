"""GB300 (sm_103a) implementation of the era-based time-symmetric block
time-step (TSBTS) N-body integrator of Kaplan & Saygin (Sec. 2-4).

Modules:
  tsbts   ctypes binding of the C ABI (include/tsbts.h), libtsbts.so
  build   nvcc build of libtsbts.so (in-tree)
  inputs  seeded synthetic Plummer / Salpeter workloads
"""
