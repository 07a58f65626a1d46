"""GB300-native optimized Schwarz solver for the gravimetry equations.

Python binding of ``libosm.so`` (C ABI in ``include/osm.h``).  The library
must be built first (``paper_2112_03851_gb300.build.build()``); importing
the solver without it raises ImportError -- there is no CPU fallback.
"""
from ._lib import (  # noqa: F401
    BatchSolver, EXPORTED, LIB_PATH, OSM_FP64, OSM_MIXED, OsmError, Solver, default_opts, gravity_misfit,
    gravity_potential, host_face_stiffness, host_face_system, host_local_system, load, log_uniform_p,
)
