"""GB300-native Joseph projector (forward and exact adjoint, non-TOF,
TOF-sinogram and TOF-listmode) after Schramm & Thielemans, PARALLELPROJ
(arXiv 2212.12519), Sec. 2.1-2.2.

The compute path is the C-ABI library ``libjoseph.so`` (hand-written CUDA
for sm_103a, declared in ``include/joseph.h``); ``ops`` is its thin ctypes
binding.  Importing this package does not load the library; the first call
into ``ops`` does, and fails loudly when it is missing.
"""
__all__ = ["ops", "synth"]
