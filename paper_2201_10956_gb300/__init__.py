"""GB300-native exhaustive three-way epistasis scan (arXiv 2201.10956 hot path).

The compute path is the CUDA library ``libepi3.so`` (C ABI in include/epi3.h);
this package holds its sources (csrc/), its build script and a ctypes binding.
"""
from .epi3 import (Batch, DEVICE_PTRS, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_OVERFLOW, ERR_TIMEOUT,
                   ERR_UNSUPPORTED, LIB_PATH, MAX_TOPK, OK, PATH_AUTO, PATH_MMA, PATH_MMA16, PATH_MMA4, PATH_MMA4C, PATH_POPC, PATH_POPC8, SYMBOLS,
                   Epi3Error, Handle, last_error, load, scan_batch)

__all__ = ["Handle", "Batch", "scan_batch", "Epi3Error", "load", "last_error", "LIB_PATH", "SYMBOLS", "MAX_TOPK",
           "PATH_AUTO", "PATH_POPC", "PATH_POPC8", "PATH_MMA", "PATH_MMA16", "PATH_MMA4", "PATH_MMA4C", "DEVICE_PTRS", "OK", "ERR_ARG", "ERR_CUDA", "ERR_OOM",
           "ERR_TIMEOUT", "ERR_UNSUPPORTED", "ERR_OVERFLOW"]
