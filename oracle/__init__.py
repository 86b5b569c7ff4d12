"""FP64 CPU oracle of the cutting voxel projector -- test infrastructure only.

Only the test-suite, the package smoke check and the benchmark's CPU-baseline leg
use this package. It shares no code with the CUDA library: the arithmetic lives in
``oracle.c`` (generic convex-polytope clipping in double precision), compiled with
gcc into ``liboracle.so`` next to it.
"""
from .oracle import *  # noqa: F401,F403
