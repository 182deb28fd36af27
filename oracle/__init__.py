"""FP64 CPU oracle for the bundle-adjustment iteration (test infrastructure).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA path.
"""
from .ba_oracle import *  # noqa: F401,F403
from . import pose_graph, priors, rig_ba, triangulation  # noqa: F401
