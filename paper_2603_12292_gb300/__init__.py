"""GB300-native population evaluation for GP symbolic regression.

The compute path is the CUDA library libsr (include/sr.h) built in-tree by
``paper_2603_12292_gb300.build``; ``binding`` is its ctypes front end.
Importing this package loads nothing; the library is loaded on first use.
"""
__all__ = ["binding", "build", "inputs"]
