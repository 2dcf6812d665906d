"""Seeded synthetic inputs for the periodic eddy-current problem on a coaxial cable.

This package is the only code shared by the CPU oracle (``oracle/``) and the GPU
path (``paper_1905_13076_gb300``).  It produces *data* only — node coordinates,
triangles, region tags, Dirichlet flags, material constants and excitation
parameters — and contains none of the method's arithmetic (no element
integrals, no time stepping, no solves).

The paper's workload is a nonlinear 2D coaxial-cable model (Sec. 4); its
geometry and materials are not given in the paper, so the structured polar
meshes generated here stand in for it.
"""

from .coax import (  # noqa: F401
    BRAUER_BMAX,
    BRAUER_STEEL,
    NU0,
    RADII,
    REGION_AIR,
    REGION_CORE,
    REGION_INSULATION,
    REGION_SHEATH,
    CoaxMesh,
    Problem,
    batched_cables,
    coax_mesh,
    make_problem,
    radial_intervals,
    workload,
    WORKLOADS,
)
