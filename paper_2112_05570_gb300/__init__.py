"""GB300-native closest-hit ray queries through constrained triangulations
(Frederickx & Dutre, arXiv 2112.05570, Sec. 5): a C-ABI CUDA library
(``include/cct.h``, built from ``csrc/``) and its thin Python binding."""
from ._build import build  # noqa: F401
from .cct import *  # noqa: F401,F403
