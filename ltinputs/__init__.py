"""Seeded synthetic inputs for the sparse lighting-matrix renderer.

This package only *creates inputs*: procedural box scenes, the shading points seen
by a pinhole camera and the virtual point lights (VPLs) deposited by one bounce of
light tracing.  It holds none of the method's arithmetic (no entry evaluation, no
visibility test between shading points and VPLs, no sampling, no completion), so
that both the CPU oracle and the CUDA path can consume the same arrays without
sharing any of the code under test.
"""
from .configs import CONFIGS, get_config
from .scenes import load_or_make_scene, make_scene, Scene

__all__ = ["CONFIGS", "get_config", "load_or_make_scene", "make_scene", "Scene"]
