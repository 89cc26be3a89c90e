"""GB300 hot path of FastFourierSAT: batched Walsh-Fourier objective and gradient.

Submodules are imported lazily: ``gen`` (seeded synthetic inputs) has no
dependency on the compiled library; ``ffsat`` is the binding to the CUDA
C-ABI library and fails loudly if that library is missing.
"""
__all__ = ["gen", "ffsat"]
