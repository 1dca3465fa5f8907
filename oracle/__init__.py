"""FP64 CPU oracle of the per-pixel ray tracer (arXiv 2305.07450, Section 3).

Test infrastructure only: tests, the package smoke check and the bench's CPU
baseline leg may import it; the product path never does.
"""
from .oracle import *  # noqa: F401,F403
