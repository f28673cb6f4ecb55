"""GB300-native differentiable Voronoi ray tracing (arXiv 2608.17682).

The CUDA library (libvt.so, C ABI in include/vt.h) is loaded lazily on first
use of ``api`` / ``_vt``: importing the package alone (e.g. for
``workloads``) needs no GPU. Using the renderer without the built library
raises ImportError -- there is no CPU fallback.
"""
import importlib

__all__ = ["api", "workloads", "build"]


def __getattr__(name):
    if name in ("api", "_vt", "workloads", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
