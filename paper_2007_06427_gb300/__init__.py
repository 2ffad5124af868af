"""GB300 (sm_103a) tau-descent of Kuramoto-Sivashinsky loops: adjoint-based variational method
of Azimi, Ashtari & Schneider (arXiv:2007.06427).

The compute path is the CUDA library ``libks_loop.so`` behind the C ABI of
``include/ks_loop.h``; ``ks_loop`` is its ctypes binding.  Submodules are imported lazily so
that the input generators can be used on machines without the library.
"""
__all__ = ["ks_loop", "inputs", "autograd", "build"]
