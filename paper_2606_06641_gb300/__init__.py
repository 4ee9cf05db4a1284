"""GB300-native Fourier-expansion continuous local search (CLS) for symmetric
pseudo-Boolean constraints.

``binding`` is the thin Python layer over the C ABI of ``include/afsat.h``
(the CUDA library built in-tree by ``build``); ``synth`` draws seeded
synthetic instances. Importing the package loads nothing: the library is
opened on first use and raises if it has not been built.
"""
__all__ = ["binding", "synth", "build"]
