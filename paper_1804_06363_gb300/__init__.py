"""GB300-native online reduced-basis solvers (RBI, RB-preconditioned CG).

The compute path is librb.so (hand-written sm_103a CUDA behind the C interface
in include/rb.h); `rb` is its ctypes binding.  Importing the package does not
load the library; the first call into `rb` does, and raises if it is missing.
"""
from . import rb  # noqa: F401
from .rb import Context, RbError  # noqa: F401
