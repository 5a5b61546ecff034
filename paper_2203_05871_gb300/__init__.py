"""GB300-native MPO Lindblad solver (Landa & Misguich, 2022): Python binding.

The product is the C-ABI library ``libmpdo.so`` (header ``include/mpdo.h``);
this package only loads it and marshals arguments (``mpdo.Solver``).
"""
from .mpdo import (FAULT_DROP_CTA, FP64, MIXED_BF16X3, MIXED_TF32, MPDO_ECAPACITY, MPDO_ENOCONV,  # noqa: F401
                   MPDO_ENONFINITE, MPDO_ETIMEOUT, MPDO_OK, ST_CAPACITY, ST_NOCONV, ST_NONFINITE, ST_TIMEOUT,
                   STORE_F32, STORE_F64, MpdoError, Solver, exported_symbols, load_library)

__all__ = ["Solver", "MpdoError", "load_library", "exported_symbols", "FP64", "MIXED_TF32", "MIXED_BF16X3",
           "STORE_F64", "STORE_F32", "FAULT_DROP_CTA", "MPDO_OK", "MPDO_ENOCONV", "MPDO_ETIMEOUT",
           "MPDO_ENONFINITE", "MPDO_ECAPACITY", "ST_NOCONV", "ST_NONFINITE", "ST_TIMEOUT", "ST_CAPACITY"]
