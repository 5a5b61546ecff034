"""GB300-native MPO Lindblad solver (Landa & Misguich, 2022): Python binding.

The product is the C-ABI library ``libmpdo.so`` (header ``include/mpdo.h``);
this package only loads it and marshals arguments (``mpdo.Solver``).
"""
from .mpdo import (FP64, MIXED_BF16X3, MIXED_TF32, STORE_F32, STORE_F64, MpdoError, Solver,  # noqa: F401
                   exported_symbols, load_library)

__all__ = ["Solver", "MpdoError", "load_library", "exported_symbols", "FP64", "MIXED_TF32", "MIXED_BF16X3",
           "STORE_F64", "STORE_F32"]
