"""Real-space / imaginary-time GW sweep (arXiv:1911.05633) on one GB300.

The compute path is libgw.so (CUDA for sm_103a, C ABI in include/gw.h); the
module ``paper_1911_05633_gb300.gw`` is its Python binding.  Build with
``python -m paper_1911_05633_gb300.build``.
"""
__all__ = ["gw", "build"]
