"""GB300-native bin-level q-gram filter (GRIM-Filter hot path).

The CUDA kernels and their C-ABI live in ``csrc/`` and ``include/grim.h``;
``grim`` is the thin ctypes binding with the same entry-point names, and
``synth`` holds the seeded synthetic-input generators.
"""
__all__ = ["grim", "synth"]
