"""GB300-native Ewald summation (arXiv 1708.01135 hot path).

``Ewald`` / ``Server`` / ``tune`` bind the C ABI of ``libewald.so`` (include/ewald.h);
``workloads`` holds the seeded synthetic inputs.  Importing the package does not load the
CUDA library; the first call does, and fails loudly if it has not been built.
"""
from .ewald import (Ewald, EwaldError, Server, tune, FP64, MIXED, MIXED_BF16, FP32,  # noqa: F401
                    PART_REAL, PART_RECIP, PART_SELF, PART_ALL, MD_RECORD, real_noalloc,
                    NOALLOC_MAX_N, fma_peak)
