"""B300-native non-subsampled digital shearlet transform (ShearLab 3D hot path).

The transform runs in hand-written sm_103a CUDA kernels behind the C ABI of
``libshearlet.so`` (see include/shearlet.h); ``paper_1402_5670_b300.shearlet``
is the thin ctypes binding over it. The native library is loaded on first use.
"""
