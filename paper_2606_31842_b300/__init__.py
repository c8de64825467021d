"""B300-native eigenvector-deflated WaveHoltz (sm_103a CUDA kernels behind a C ABI).

    from paper_2606_31842_b300 import whv      # ctypes binding of include/whv.h (needs libwhv.so)
    from paper_2606_31842_b300 import inputs   # seeded synthetic workloads (no method arithmetic)

The binding is not imported here so that the input generators stay importable on machines
without the built library.
"""
__all__ = ["whv", "inputs", "build"]
