"""FP64 CPU oracle for the L1 IRLS + PCG phase-unwrapping path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline and reference
legs) may import this package.  The product path (the CUDA library and its Python binding)
never imports it, and this package imports nothing from the product.
"""
from .irls import *  # noqa: F401,F403
from .irls import __all__  # noqa: F401
