"""Seeded synthetic inputs (scenes, sequences, batches) for the pose-graph
library, its tests and its benchmark.  Holds no pose-graph arithmetic."""
from .scene import *  # noqa: F401,F403
from .sequence import Sequence, paper_sequence  # noqa: F401
