"""FP64 CPU oracle of the particle-resolved thermal LBM step (arXiv 2308.16597).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
CPU-baseline leg of the benchmark, never by the package's product path.  It
shares no code with the CUDA library.
"""
from .oracle import Oracle, build, load, ORC_PARTICLE_DTYPE  # noqa: F401
