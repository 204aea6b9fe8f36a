"""Seeded synthetic inputs (scenes, sequences, batches) for the pose-graph
library, its tests and its benchmark.  Holds no pose-graph arithmetic."""
from .scene import *  # noqa: F401,F403
