"""GB300-native score-only Smith-Waterman/Gotoh with the striped max-plus
scan of F (arXiv:1909.00899, Alg. 6) and the lazy-F comparison (Alg. 1).

The compute path is the C-ABI library ``libsw_gb300.so`` (hand-written
sm_103a CUDA); :mod:`paper_1909_00899_gb300.sw` is its thin ctypes binding.
Importing the package loads nothing; the binding loads the library on first
use and raises if it is missing.  There is no CPU fallback.
"""
__all__ = ["sw", "synth"]
