"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This package only *generates inputs*: triangle meshes, per-triangle and
per-instance materials, camera and instance keyframes, and environment-map
texels, and event videos for the quality metrics.  It holds none of the method's arithmetic (no ray tracing, no
statistics, no sampling of paths).  Every function is deterministic in its
`seed` argument.
"""
from .procedural import (  # noqa: F401
    Scene,
    Workload,
    WORKLOADS,
    albedo_texture,
    textured_room,
    BATCH_RESOLUTIONS,
    batch_workloads,
    cornell_box,
    empty_env,
    event_video_pair,
    furnace_sphere,
    icosphere_field,
    plane_under_env,
    textured_plane,
    sky_texture,
    static_variant,
    terrain_with_boxes,
    workload,
)
