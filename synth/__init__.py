"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package only draws inputs: surface triangulations (geodesic spheres,
ellipsoids, cubes) with seeded vertex jitter, and plane-wave excitations.  It
holds none of the method's arithmetic (no basis functions, no quadrature, no
operators), so both the CPU oracle and the GPU path may import it.
"""

from .meshes import (  # noqa: F401
    Mesh,
    geodesic_sphere,
    ellipsoid,
    cube,
    torus,
    plate,
    open_cylinder,
    mesh_for_config,
)
from .excitation import (  # noqa: F401
    plane_wave_z,
    random_plane_waves,
)
