"""Seeded synthetic inputs shared by the oracle-side tests and the GPU path.

This package only produces inputs: mesh coordinates, per-element density
anomalies, subdomain cut positions, station positions and sampled Robin
parameters.  It contains none of the method's arithmetic (no assembly, no
solver, no transmission update).
"""
from .workloads import *  # noqa: F401,F403
