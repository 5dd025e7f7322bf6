"""GB300-native (sm_103a) staggered-grid Fourier pseudo-spectral elastic
seismogram simulator after Das, Chen & Hobson (arXiv 1705.04874).

The solver is the C-ABI library ``libes.so`` (hand-written CUDA); ``es`` is
its thin ctypes binding, ``synth`` the seeded synthetic-input generators."""
__all__ = ["es", "synth"]
