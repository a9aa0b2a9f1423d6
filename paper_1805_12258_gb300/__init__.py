"""GB300-native harmonic summing for Fourier-domain acceleration search.

The compute path is the CUDA library ``libhs.so`` (C ABI in ``include/hs.h``);
``paper_1805_12258_gb300.hs`` is its thin ctypes binding and
``paper_1805_12258_gb300.synth`` draws seeded synthetic inputs.  Importing the
package loads nothing; the binding loads the library on first use and raises
if it is missing.
"""
__all__ = ["hs", "synth"]
