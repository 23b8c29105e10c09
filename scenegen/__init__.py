"""Seeded synthetic input generator for the constraint-resolution hot path.

Builds tetrahedral FE meshes, the implicit system matrix, a nested-dissection
supernodal LDL^T factor of it and contact scenes.  It is the one module both
the GPU library's tests and the FP64 oracle's tests consume; it holds none of
the constraint-resolution arithmetic (no W_H, W, PGS or corrective motion).
"""
from .scenes import NAMED, Scene, batch_scenes, batch_specs, beam_scene, ellipsoid_scene, press_scene  # noqa: F401
