"""GB300 (sm_103a) OFDM monostatic radar receive chain.

The CUDA library libofdm_radar.so (include/ofdm_radar.h) implements the
chain of arXiv 2209.03883; `radar` is its thin ctypes binding.  Importing
`paper_2209_03883_gb300.radar` fails loudly when the library is not built.
"""
