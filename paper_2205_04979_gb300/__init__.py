"""GB300-native particle-deposition path: libpdq (CUDA, sm_103a) behind a C ABI.

``pdq`` is the thin ctypes binding of include/pdq.h.  Importing the package
does not build anything; ``paper_2205_04979_gb300.build.build()`` compiles
libpdq.so in-tree.
"""
from . import pdq  # noqa: F401
