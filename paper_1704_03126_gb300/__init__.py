"""GB300-native discrete velocity method for the steady linearized BGK equation.

The solver behind a C-ABI library (``libdvm.so``, declared in ``include/dvm.h``) with a thin
ctypes binding in :mod:`paper_1704_03126_gb300.dvm`.  Submodules are imported lazily so that the
input generators can be used without the CUDA library.
"""
__all__ = ["dvm", "inputs", "autograd"]
