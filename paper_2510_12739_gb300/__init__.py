"""GB300-native CoNet-Rx hot path: CUDA kernels for sm_103a behind the libconet C ABI.

``paper_2510_12739_gb300.api`` is the Python binding; importing it loads
``libconet.so`` and raises ImportError when the library has not been built.
"""
from ._lib import ConetError, LIB_PATH, lib  # noqa: F401

__all__ = ["ConetError", "LIB_PATH", "lib"]
