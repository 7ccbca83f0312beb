"""GB300-native event-parallel NLO matrix elements (arXiv:2503.07439 hot path).

Thin Python binding over the C ABI declared in ``include/me.h``: argument marshalling
only.  Every step of the computation runs in the CUDA library ``libme_gb300.so``;
there is no CPU fallback -- importing the binding without the built library, or
calling it without a CUDA device, raises.
"""
from ._capi import (ME_ERR_ARG, ME_ERR_BUSY, ME_ERR_CUDA, ME_ERR_OOM, ME_ERR_PROCESS, ME_ERR_TIMEOUT,
                    ME_OK, ME_PARAMS_VERSION, ME_PREC_FP64, ME_PREC_MIXED, ME_RESCUE_ITEMS, ME_RESCUE_POINTS,
                    ME_TERMS_AUTO, ME_TERMS_MASKED, ME_TERMS_QUEUED, MEError, Handle, Server, declared_symbols,
                    default_params, library, load_library)

__all__ = ["Handle", "Server", "MEError", "default_params", "load_library", "library", "declared_symbols",
           "ME_OK", "ME_ERR_ARG", "ME_ERR_OOM", "ME_ERR_PROCESS", "ME_ERR_TIMEOUT", "ME_ERR_CUDA",
           "ME_ERR_BUSY", "ME_PREC_FP64", "ME_PREC_MIXED", "ME_RESCUE_ITEMS", "ME_RESCUE_POINTS",
           "ME_PARAMS_VERSION", "ME_TERMS_MASKED", "ME_TERMS_QUEUED", "ME_TERMS_AUTO"]
