"""GB300-native layer editing on UV-indexed textures (arXiv 2501.14807).

The compute path is the CUDA library ``liblcl.so`` (C ABI in include/lcl.h); ``lcl``
is its thin Python binding and ``build`` compiles it for sm_103a.
"""
from . import build, lcl  # noqa: F401
