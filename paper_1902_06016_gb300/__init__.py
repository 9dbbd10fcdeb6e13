"""GB300-native IP-GFCC linear systems with model-order reduction (arXiv 1902.06016).

The computation lives in ``libgfcc.so`` (CUDA, sm_103a) behind the C ABI of ``include/gfcc.h``;
``gfcc.Context`` is its thin Python binding. ``build.build()`` compiles the library in-tree.
"""
from .gfcc import Context, GfccError, load, PRECISIONS  # noqa: F401
