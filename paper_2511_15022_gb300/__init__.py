"""GB300-native (sm_103a) hot path of complex-valued 2D Gaussian hologram optimisation
(arXiv 2511.15022): tile-binned complex rasteriser, band-limited angular spectrum
propagation with hand-written FFT passes, multi-plane intensity loss and the full
backward pass, behind the C-ABI library ``libcgh`` (see ``include/cgh.h``).

Importing the package is cheap; the CUDA library is loaded on first use by
``paper_2511_15022_gb300.cgh`` and raises if it is missing -- there is no CPU fallback.
"""
__all__ = ["inputs"]
