"""FP64 CPU oracle of the TCTF2R iteration -- test infrastructure.

Only the tests, ``__graft_entry__.smoke`` and the CPU-baseline legs of
``bench.py`` import this package.  The CUDA library never does.
"""
from . import method  # noqa: F401
from .method import *  # noqa: F401,F403
