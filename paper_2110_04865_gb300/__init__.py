"""GB300 minimum spanning forest library (algebraic Awerbuch-Shiloach).

The computation lives in the CUDA library ``_build/libmsf.so`` (C ABI in
``include/msf.h``); this package is its thin Python binding.  Build the
library with ``paper_2110_04865_gb300.build_lib.build()``.
"""
from . import _abi  # noqa: F401
from ._abi import (MSF_F32, MSF_U32, MsfError, OPT_BLOCKS_PER_SM, OPT_COMPACT_TAU,  # noqa: F401
                   OPT_JUMP_LIMIT, OPT_ROUND_LIMIT, OPT_SLOTS_PER_LANE)


def __getattr__(name):
    # the torch-facing layer is imported lazily so that the ABI can be
    # inspected without importing torch
    if name in ("Graph", "compute", "compute_batched", "Batch", "MSFWeight", "msf_weight",
                "set_option", "get_option"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
