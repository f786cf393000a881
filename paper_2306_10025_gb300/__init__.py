"""GB300-native compressed patch-based relaxation (Harper & Tuminaro,
arXiv 2306.10025): patch extraction, batched inverses, the spectral patch
criterion with Alg. 1, the additive Schwarz / Vanka sweep and the outer
Krylov solve, all in CUDA kernels behind the C ABI of include/psr.h.

This package is the thin Python binding (ctypes) of that library."""
from .binding import (Context, PsrError, load, make_opts, psr_setup, psr_extract, psr_kernel_launches,
                      psr_batched_inverse, psr_criterion, psr_spectral_norm, exported_symbols,
                      psr_setup_seeded, psr_features, MLP, psr_criterion_noalloc,
                      psr_setup_kmeans, psr_release_cached_memory, psr_memory_in_use, psr_detect_patches,
                      psr_boundary_classes, psr_setup_learned, psr_debug_inject, LIB_PATH)

__all__ = ["Context", "PsrError", "load", "make_opts", "psr_setup", "psr_extract", "psr_kernel_launches",
           "psr_batched_inverse", "psr_criterion", "psr_spectral_norm", "exported_symbols",
           "psr_setup_seeded", "psr_features", "MLP", "psr_criterion_noalloc",
           "psr_setup_kmeans", "psr_release_cached_memory", "psr_memory_in_use", "psr_detect_patches",
           "psr_boundary_classes", "psr_setup_learned", "psr_debug_inject", "LIB_PATH"]
