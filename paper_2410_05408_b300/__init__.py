"""B300-native oblate-planet transit light curves (arxiv 2410.05408).

The compute path is the CUDA library ``libgl.so`` (sources in ``csrc/``, C-ABI in
``include/gl.h``); ``binding`` marshals arguments to it through ctypes.  Importing
this package loads nothing; ``binding`` loads the library on first use and
raises if it is missing.
"""
__all__ = ["binding", "inputs"]
