"""GB300-native TPC track-model decoding (arXiv:2411.02206, Sec. 4).

The decoder is the C-ABI library ``libtmd.so`` (hand-written CUDA for sm_103a);
``paper_2411_02206_gb300.tmd`` is its ctypes binding and ``synth`` the seeded
generator of synthetic compressed frames.  Importing the package loads nothing.
"""
