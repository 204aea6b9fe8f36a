"""Seeded synthetic inputs (scenes, sequences, batches) for the pose-graph
library, its tests and its benchmark.  Holds no pose-graph arithmetic."""
from .scene import *  # noqa: F401,F403
from .sequence import Sequence, paper_sequence  # noqa: F401
from .training import (HELDOUT_SEED, TRAIN_SEED, WARMSTART_LAYERS, TrainingPool, training_graph,  # noqa: F401
                       training_graphs, warmstart_init)
