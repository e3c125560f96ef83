"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This package holds no arithmetic of the collision-detection method: it builds
meshes (subdivided icospheres with radial bumps), random rigid poses and pair
lists.  Both the FP64 oracle and the CUDA path consume its output unchanged.
"""
from .icosphere import (  # noqa: F401
    icosphere, bumped_icosphere, random_quaternion, quat_to_matrix_f64,
    support, Scene, scene_pairs, scene_c1, scene_c2, scene_c3, scene_tiny, scene_regular_pair,
    scene_particle_on_plane, scene_packing, scene_disparity, scene_regular_disparate_pair,
    scene_chain,
)
