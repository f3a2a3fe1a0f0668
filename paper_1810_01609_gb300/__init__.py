"""GB300-native (sm_103a) even-odd preconditioned Moebius domain-wall fermion propagator
solver (arXiv:1810.01609): a C-ABI library (libmdwf.so, include/mdwf.h) of hand-written
CUDA kernels, with this thin Python binding.  There is no CPU fallback: importing the
binding's functions loads the compiled library and fails if it is missing."""
from ._lib import *  # noqa: F401,F403
from ._lib import load, MdwfError, PRECS, OP, OPS  # noqa: F401
from .api import Context  # noqa: F401

load()
