"""GB300-native LRBMS online time step for two-phase flow (arXiv 1405.2810).

The compute lives in liblrbms.so (CUDA, sm_103a) behind the C ABI of
include/lrbms.h; ``lrbms`` is its ctypes binding and ``build`` compiles it.
"""
from . import lrbms  # noqa: F401
from .lrbms import *  # noqa: F401,F403
