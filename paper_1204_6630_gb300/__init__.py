"""GB300-native brute-force angular pair counting (DD, DR, RR) and the
Landy-Szalay estimator w(theta).

The computation lives in ``libtpcf.so`` (CUDA kernels for sm_103a and a C++
host runtime behind the C ABI of ``include/tpcf.h``).  ``tpcf`` is its ctypes
binding, ``build`` compiles it, ``synth`` generates seeded synthetic catalogs.
Submodules are imported on demand so that ``synth`` works without the CUDA
library.
"""
import importlib

__all__ = ["tpcf", "build", "synth"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
