"""Seeded synthetic inputs shared by the tests, the oracle checks and bench.py.

Holds no arithmetic of the segmentation method itself."""
from .cubes import WORKLOADS, Workload, make, random_cube, voronoi  # noqa: F401
