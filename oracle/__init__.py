"""FP64 CPU oracle for the hex8 element assembly path (test infrastructure only).

Only tests, the package smoke check and the bench's CPU-baseline leg may import this
package.  It shares no code with the CUDA library; the two meet only through the seeded
inputs of `paper_2604_22087_b300.inputs`.
"""
from .fem import *  # noqa: F401,F403
from . import mlp  # noqa: F401
