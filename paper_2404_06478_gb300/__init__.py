"""GB300-native (sm_103a) hot path of LaueOT Sinkhorn-EM indexing.

The compute path is liblaueot.so (hand-written CUDA behind the C ABI in
include/laueot.h); ``api`` is its thin Python binding.  Importing the package
does not load the library; ``build.build()`` compiles it in-tree.
"""

__all__ = ["api", "build"]
