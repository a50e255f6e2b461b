"""GB300-native short-range PP gravity (PM-split factor, Plummer softening,
hard cutoff, periodic box) over octree leaf-pair lists.

The compute lives in libphpp.so (include/phpp.h, sources in csrc/); the
``binding`` module is a thin ctypes layer with the same names as the C ABI,
and ``synth`` draws the seeded synthetic particle sets.
"""
__all__ = ["binding", "synth"]
