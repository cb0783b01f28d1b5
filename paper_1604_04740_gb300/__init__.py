"""GB300-native numerical entanglement: exact fault-tolerant integer GEMM and
circular convolution on M entangled streams (Anam & Andreopoulos).

The compute path is the CUDA library libne.so (C ABI in include/ne.h); the
binding is `paper_1604_04740_gb300.ne`.  Importing the binding builds/loads
the library and fails loudly if it cannot.
"""
import importlib

__all__ = ["ne", "inputs"]


def __getattr__(name):
    if name in ("ne", "inputs", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
