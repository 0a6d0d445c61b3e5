"""GB300 short-range non-bonded library (cluster pair algorithm, arXiv:2006.09167).

The compute path is libnb.so (hand-written CUDA for sm_103a behind the C ABI
of include/nb.h); this package is its Python binding.  Importing
`paper_2006_09167_gb300.api` loads the library and fails if it is not built.
"""
__all__ = ["api", "build", "synth"]
