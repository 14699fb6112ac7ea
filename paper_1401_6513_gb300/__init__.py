"""GB300 (sm_103a) path of the virtual interpolation point fractional-step solver.

Park, Jo and Choe, "Virtual Interpolation Point Method for Viscous Flows in
Complex Geometries" (arXiv:1401.6513).  The method runs in libvip.so (CUDA,
C ABI declared in include/vip.h); ``vip`` is its ctypes binding.
"""
from .build import build  # noqa: F401


def load():
    """Import the binding (raises ImportError if libvip.so has not been built)."""
    from . import vip
    vip.lib()
    return vip
