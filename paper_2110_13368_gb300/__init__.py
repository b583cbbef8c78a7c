"""GB300-native LOD substrate transport step (diffusion, decay, cell sources)
of the hybrid agent-based model of Eq. 1 (arXiv 2110.13368), behind the C ABI
of include/bfvm.h.

Import is light: the compiled library is loaded on first use of
``paper_2110_13368_gb300.bfvm``.
"""
__all__ = ["bfvm", "inputs", "build"]
