"""GB300-native deterministic hypergraph coarsening and label propagation
(the data-parallel core of Mt-KaHyPar's deterministic multilevel
partitioner, arXiv 2303.17679).

The compute path is libhg.so (hand-written sm_103a CUDA behind the C ABI in
include/hg.h); ``hg`` is its thin ctypes binding.
"""
from . import hg  # noqa: F401

__all__ = ["hg"]
