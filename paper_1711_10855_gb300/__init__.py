"""GB300-native FDAS correlation: the overlap-and-save f-fdot power plane (arXiv 1711.10855).

The compute path is the C-ABI library ``libfdas.so`` (hand-written sm_103a CUDA under
``csrc/``, declared in ``include/fdas.h``).  ``fdas`` is its thin ctypes binding; ``synth``
makes seeded synthetic input spectra.  Importing this package loads nothing: the library is
loaded on first use by ``fdas.lib()`` and raises if it is missing.
"""
__all__ = ["fdas", "synth"]
