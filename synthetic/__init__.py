"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module draws geometry and random numbers only: tetrahedral meshes of the
imaging chamber (Section 1: metallic cylinder of diameter 28.5 cm and height
28 cm, here radius 0.15 m as the workloads state), relative permittivity maps
sampled at tet centroids, antenna positions and the Gaussian draws used to add
noise to synthetic measurements (Section 6.3).  It holds none of the method's
arithmetic (no finite elements, no solver, no misfit), so both sides of every
parity test can take their inputs from here without sharing code.
"""

from .mesh import kuhn_box_mesh, cube_mesh, chamber_mesh, Mesh
from .maps import (
    EPS_GEL,
    EPS_HEAD,
    EPS_BLOOD_LIKE,
    EPS_LOW,
    cube_eps,
    chamber_eps,
    chamber_target_eps,
    tet_centroids,
)
from .antennas import Antenna, cube_antennas, ring_antennas, antenna_array
from .noise import noise_draws, add_noise

__all__ = [
    "Mesh", "kuhn_box_mesh", "cube_mesh", "chamber_mesh",
    "EPS_GEL", "EPS_HEAD", "EPS_BLOOD_LIKE", "EPS_LOW",
    "cube_eps", "chamber_eps", "chamber_target_eps", "tet_centroids",
    "Antenna", "cube_antennas", "ring_antennas", "antenna_array",
    "noise_draws", "add_noise",
]
