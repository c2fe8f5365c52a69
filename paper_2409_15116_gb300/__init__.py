"""GB300-native DMPT/TDA Bethe-Salpeter hot path: C-ABI CUDA library + thin Python binding.

The compute runs in ``_lib/libbse.so`` (built by ``build.build()``); ``binding`` only
marshals arguments. See ``include/bse.h`` for the ABI.
"""
from .binding import (Context, BseError, load, version, PREC_FP64, PREC_MIXED,  # noqa: F401
                      EXPORTS, LIB_PATH)
