"""Seeded synthetic inputs shared by the CUDA library's tests, the benchmark
and the oracle.  Holds no beamforming arithmetic."""
from . import scenes  # noqa: F401
