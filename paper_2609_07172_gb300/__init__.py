"""Batched Fourier-mode multigrid field solve for cylindrical PIC, on GB300.

The solver itself is the C-ABI CUDA library declared in include/pic_poisson.h
(built from csrc/ by :mod:`.build`); :mod:`.binding` marshals PyTorch tensors
into it, and :mod:`.workloads` draws the seeded synthetic inputs.
"""
from .binding import (FP64, MIXED, BatchPlan, Plan, PicPoissonError, autotune, cell_coeffs, last_error, load,
                      measure_fma_peaks, query)

__all__ = ["FP64", "MIXED", "BatchPlan", "Plan", "PicPoissonError", "autotune", "cell_coeffs", "last_error", "load",
           "measure_fma_peaks", "query"]
