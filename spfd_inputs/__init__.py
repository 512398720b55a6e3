"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This package only *generates inputs*: voxel conductivity phantoms, edge
vector potentials of analytic magnetic sources and facet fluxes of their
closed-form flux densities (``flux.py``).  It holds none of the arithmetic of
the SPFD method itself (no conductance averaging, no gradient or curl, no
Poisson operator, no solver, no gauging, no field evaluation).

Grid conventions (used by every consumer):

* voxels ``(i, j, k)`` are the primary cells; arrays are indexed
  ``[k][j][i]`` (z slowest, x fastest), shape ``(nz, ny, nx)``;
* nodes sit at voxel corners, node grid ``(nz+1, ny+1, nx+1)``;
  node ``(i, j, k)`` is at ``(i*h - ox, j*h - oy, k*h - oz)``;
* the d-directed edge stored at node ``(i, j, k)`` runs from that node to the
  next node along axis d; edge arrays have shape ``(3, nz+1, ny+1, nx+1)``
  with component 0/1/2 = x/y/z edges; slots past the last node along the
  edge's own axis do not correspond to an edge and are zero.
"""

from .phantoms import (
    BODY_ELLIPSOIDS,
    Phantom,
    body_phantom,
    random_phantom,
    scaled_body_phantom,
    sphere_phantom,
)
from .flux import loop_flux, loop_flux_density, uniform_flux
from .sources import (
    MU0,
    edge_potential,
    loop_potential,
    loop_vector_potential,
    random_loops,
    uniform_b_landau,
    uniform_b_symmetric,
)

__all__ = [
    "BODY_ELLIPSOIDS",
    "Phantom",
    "body_phantom",
    "random_phantom",
    "scaled_body_phantom",
    "sphere_phantom",
    "MU0",
    "edge_potential",
    "loop_flux",
    "loop_flux_density",
    "uniform_flux",
    "loop_potential",
    "loop_vector_potential",
    "random_loops",
    "uniform_b_landau",
    "uniform_b_symmetric",
]
