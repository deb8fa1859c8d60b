"""Seeded synthetic inputs (meshes, initial states) shared by the oracle and
the CUDA library tests/benchmarks.  Holds none of the method's arithmetic."""
from . import meshes, states  # noqa: F401
