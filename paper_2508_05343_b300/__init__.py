"""B300-native (sm_103a) 3D Gabor splatting rasterizer: C-ABI library plus a thin Python binding.

Submodules are loaded lazily so that the seeded input generator (``scenes``) can be imported
without loading the CUDA library.
"""
import importlib

__all__ = ["scenes", "binding", "raster", "serve", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
