"""GB300 (sm_103a) implementation of Fox / LazyFox overlapping community
detection (Garrels et al., arXiv 2210.03211): hand-written CUDA kernels behind
the C ABI of ``include/lazyfox.h``, with a thin Python binding.

The CUDA library is loaded on first use (``lazyfox.load_library``); without it
every call raises -- there is no CPU fallback.
"""
from .lazyfox import (ABI_FUNCTIONS, Batch, Graph, Server, cover_f1, quality_report, LazyFoxError, RunStats, load_library,  # noqa: F401
                      run_lazyfox)

__all__ = ["Batch", "Graph", "Server", "cover_f1", "quality_report", "LazyFoxError", "RunStats", "load_library", "run_lazyfox", "ABI_FUNCTIONS"]
