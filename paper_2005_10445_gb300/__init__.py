"""GB300-native acquisition-mode time-of-arrival search (coherent code x
carrier-offset search with fused on-chip FFT correlation).

``synth`` makes seeded synthetic inputs; ``binding`` is the thin ctypes
layer over the C-ABI library ``libatlas_acq.so`` built from ``csrc/``.
The binding is imported lazily so that input generation does not require
the compiled library.
"""

__all__ = ["synth", "binding"]
