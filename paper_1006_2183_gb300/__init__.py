"""GB300-native semiring SpGEMM (C = A*B) with a 2D virtual Sparse SUMMA grid.

The compute path lives in the CUDA library ``libspgemm.so`` (sources under
``csrc/``, C-ABI declared in ``include/spgemm.h``); ``spgemm`` is its ctypes
binding.  ``gen`` holds the seeded synthetic input generators.  Importing the
package does not load the CUDA library; ``from paper_1006_2183_gb300 import
spgemm`` does, and fails loudly if it is missing.
"""
__all__ = ["gen", "spgemm"]
