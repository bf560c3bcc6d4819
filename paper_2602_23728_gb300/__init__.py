"""GB300-native three-phonon scattering (kALDo 2.0 hot path): Python binding of libphx.

The compute lives in the CUDA library libphx.so (built by paper_2602_23728_gb300.build);
this package only marshals arguments.  Importing it without the built library raises.
"""
from ._lib import (Context, FC3, PhxError, irreducible, time_reversal_count, version, EXPORTED, LIB_PATH,  # noqa: F401
                   PHX_FP64, PHX_TF32, PHX_BF16X3, kappa_rta_noalloc)
