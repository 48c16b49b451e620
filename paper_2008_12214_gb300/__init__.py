"""GB300-native iterative Fourier-transform hologram engine (GS, WGS, OSPR).

The compute path is the C-ABI library ``libhologen.so`` (hand-written sm_103a
CUDA); ``paper_2008_12214_gb300.hologen`` is its thin ctypes binding.
"""
