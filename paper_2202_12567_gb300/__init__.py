"""Sparse sampling and completion of the VPL lighting matrix on GB300 (sm_103a).

``lt`` is the thin binding of the C-ABI library liblt.so (include/lt.h);
``renderer.Renderer`` owns the tensors of one scene and runs frames through it.
Importing a submodule that touches the library fails loudly if liblt.so has not
been built (``build.build()``).
"""
__all__ = ["lt", "renderer", "build"]
