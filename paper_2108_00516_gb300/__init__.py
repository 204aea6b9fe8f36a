"""GB300 (sm_103a) implementation of BundleTrack's online pose-graph
optimisation (Wen & Bekris, IROS 2021, Sec. IV-D), behind the C interface in
include/bt.h.  ``bt`` is the Python binding of that interface."""
from . import bt  # noqa: F401
from .bt import PoseGraph, graph_from_synth  # noqa: F401

__all__ = ["bt", "PoseGraph", "graph_from_synth"]
