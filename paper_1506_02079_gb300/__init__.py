"""emfuse: GB300-native gradient-domain colour correction of EM image stacks.

Kazhdan et al., "Gradient-Domain Fusion for Color Correction in Large EM Image Stacks"
(arXiv 1506.02079): anisotropic smoothing of a registered stack along z (Sec. 3
"Anisotropic Smoothing"), then one screened-Poisson solve per xy-slice, Eq. (1).

The compute lives in ``libemfuse.so`` (hand-written CUDA for sm_103a behind a C ABI, see
``include/emfuse.h``); ``paper_1506_02079_gb300.api`` is a thin binding with the same names.
The library is loaded on first use and a missing library is an error, never a fallback.
"""
__all__ = ["api", "synthetic"]
