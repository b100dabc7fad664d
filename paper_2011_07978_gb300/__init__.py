"""GB300-native batched stiff-chemistry step (DLBFoam's hot path on one GPU).

`dlbchem` is the ctypes binding of libdlbchem.so, whose C ABI is declared in
include/dlbchem.h. Build the library with `paper_2011_07978_gb300.build.build()`.
"""
from . import dlbchem  # noqa: F401
from .dlbchem import Context, options_default  # noqa: F401
