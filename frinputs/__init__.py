"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds mesh generators (nodes, connectivity, periodic vectors,
boundary faces) and closed-form initial states evaluated at given physical
points.  It contains none of the FR method's arithmetic: no point sets, no
operators, no fluxes.  Both the oracle and the CUDA library consume its
output; neither is imported here.
"""
from .meshes import box_hex, curved_box_hex, curved_mixed_box, mixed_box, MeshSpec  # noqa: F401
from . import ics  # noqa: F401
