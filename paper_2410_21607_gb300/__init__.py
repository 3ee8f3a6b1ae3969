"""GB300-native spectral-element hot path of arXiv 2410.21607 (AMR tropical cyclones).

The compute lives in libsem.so (CUDA, sm_103a) behind the C ABI of
include/sem.h; `paper_2410_21607_gb300.sem` is its ctypes binding.  Building:
`paper_2410_21607_gb300.build.build()`.
"""
