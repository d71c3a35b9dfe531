"""GB300-native spectral stepper for the Sivashinsky-type expanding-flame model
(Karlin, "Global communications in multiprocessor simulations of flames").

The compute path is the sm_103a CUDA library behind the C ABI declared in
include/flame.h; ``paper_0911_2889_gb300.flame`` is its thin ctypes binding.
Importing this package loads nothing; the library is loaded on first use.
"""
__all__ = ["flame", "inputs"]
