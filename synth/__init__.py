"""Seeded synthetic inputs for the layered Gaussian-splatting rasterizer.

This package only draws random numbers and builds camera poses.  It holds
none of the rendering arithmetic, so both the FP64 oracle (``oracle/``) and
the CUDA path (``paper_2410_16978_gb300``) can be fed from it without sharing
any of the method's code.
"""
from .scenes import (  # noqa: F401
    Camera,
    Scene,
    look_at_camera,
    stereo_pair,
    fibonacci_cameras,
    random_clip_planes,
    scene_c1,
    scene_c2,
    scene_c3,
    scene_c4,
    shell_scene,
    uniform_scene,
    config_seed,
    to_half_storage,
    from_half_storage,
)
