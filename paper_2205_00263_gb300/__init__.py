"""GB300-native batched bounding of MN-BaB branch-and-bound subproblems.

The compute path lives in ``libmnbab.so`` (hand-written sm_103a kernels behind
the C ABI of ``include/mnbab.h``); ``api`` marshals arguments to it.  There is
no CPU fallback: importing the API without the built library raises.
"""
from .api import Context, MnbabError, NodeParams  # noqa: F401
from . import _lib  # noqa: F401

VERIFIED, FALSIFIED, UNKNOWN = 1, -1, 0
