"""GB300-native eddy-current finite-element solver (A-V potentials, P1 tets).

The compute path lives in the CUDA library libect.so (C ABI in include/ect.h);
`ect` is its Python binding.  Build the library with `build.build()`.
"""
from . import build  # noqa: F401
from .ect import (ECT_DEFECT, ECT_F32, ECT_F64, ECT_MODE_F64, ECT_MODE_MIXED,  # noqa: F401
                  ECT_VACUUM, Context, EctError, default_options, load_library)
