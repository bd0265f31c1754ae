"""GB300-native Rejection-Free Partial Neighbor Search (arXiv 2210.10513).

The sampler lives in a C-ABI shared library (libpns.so, CUDA for sm_103a);
`paper_2210_10513_gb300.pns` is its thin ctypes binding.  Import it
explicitly; importing this package loads nothing.
"""
__all__ = ["pns", "synth"]
