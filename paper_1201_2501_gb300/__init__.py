"""GB300-native sparse FFT (Hassanieh, Indyk, Katabi, Price, "Nearly Optimal Sparse Fourier Transform").

The compute path is ``libsfft.so`` (hand-written sm_103a CUDA behind a C ABI, declared in
``include/sfft.h``); ``sfft`` is its thin ctypes binding.  ``workloads`` draws the seeded synthetic
inputs.  Importing the package does not load the library; the first call into ``sfft`` does, and it
raises if the library is missing.
"""
__all__ = ["sfft", "workloads"]
