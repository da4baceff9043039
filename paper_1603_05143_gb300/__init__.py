"""GB300-native per-atom Polyhedral Template Matching.

Larsen, Schmidt & Schiotz, "Robust Structural Identification via Polyhedral
Template Matching".  Every step of the per-atom method runs in the CUDA library
``libptm.so`` (C ABI in ``include/ptm.h``); this module only marshals
arguments.  PyTorch provides device memory and streams.

    from paper_1603_05143_gb300 import PTM
    ptm = PTM(device=0)
    out = ptm.classify(positions_cuda, cell)          # dict of CUDA tensors

There is no CPU fallback: if the library is missing or no GPU is present the
calls raise.
"""
from .binding import (PTM, PTMError, Batch, Server, load, measure_fma_peak, STRUCTURES, ALLOYS, MASK_ALL, MASK_SC, MASK_FCC, MASK_HCP,
                      MASK_ICO, MASK_BCC)

__all__ = ["PTM", "PTMError", "Batch", "Server", "load", "measure_fma_peak", "STRUCTURES", "ALLOYS", "MASK_ALL", "MASK_SC", "MASK_FCC",
           "MASK_HCP", "MASK_ICO", "MASK_BCC"]
