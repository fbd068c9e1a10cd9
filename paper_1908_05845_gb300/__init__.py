"""GB300-native SMMO heap and parallel_do (thesis: Springer, "Memory-Efficient
Object-Oriented Programming on GPUs", arXiv 1908.05845).

The compute path is the CUDA library ``libsmmo.so`` (sources in ``csrc/``,
C ABI in ``include/smmo.h``).  ``paper_1908_05845_gb300.smmo`` is the thin
ctypes binding; it raises if the library has not been built.  Nothing here
falls back to the CPU.
"""
__all__ = ["inputs", "smmo"]
