"""Batched spectral estimation of THz-TDS traces on GB300 (sm_103a).

Zero-padded FFT, chirp-z transform and Zoom FFT (arXiv 2108.03948) as
hand-written CUDA kernels behind a C-ABI shared library.  ``synth`` draws the
seeded synthetic traces; the transforms are exposed by the ctypes binding in
``spec`` (loaded on first use).
"""
