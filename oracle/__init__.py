"""FP64 CPU oracle of the envelope-tracking particle step.

TEST INFRASTRUCTURE: only the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this package.  It shares no code with the CUDA
library (`paper_2208_12795_gb300`) and never imports it.
"""
from .oracle import OracleMesh, build_oracle, push_step  # noqa: F401
