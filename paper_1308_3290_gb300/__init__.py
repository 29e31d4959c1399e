"""GB300-native coarse grid projection (CGP) time step for quasigeostrophic
ocean basins (San & Staples, arXiv 1308.3290).

The compute path is the C-ABI library ``libqgcgp.so`` (hand-written sm_103a
CUDA); ``paper_1308_3290_gb300.qg`` is its thin ctypes binding.  Importing
this package does not load the library: the first call that needs it does,
and raises if it is missing.
"""
__all__ = ["qg", "inputs"]
