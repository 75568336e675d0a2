"""GB300-native direct-summation N-body force + jerk with a Hermite-4
block-step integrator (libnbody.so behind a C ABI, include/nbody.h).

``NBody`` and the other binding names load the compiled library on first
use; importing the package itself loads nothing.
"""

__all__ = ["NBody", "NBodyError", "load", "variant_info", "num_variants"]


def __getattr__(name):
    if name in __all__:
        from . import _lib

        return getattr(_lib, name)
    raise AttributeError(name)
