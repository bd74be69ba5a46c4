"""GB300-native transposition of multigraphs and high-cardinality sparse
matrices (XCSR).  The compute path is the CUDA library libmgt.so (C ABI in
include/mgt.h); ``mgt`` is its Python binding."""
from . import mgt  # noqa: F401

__all__ = ["mgt"]
