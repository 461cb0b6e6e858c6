"""GB300-native all-at-once sparse triple product C = P^T A P.

``ptap`` is the binding of the CUDA library (include/ptap.h); ``problems``
builds seeded synthetic inputs; ``autotune`` picks launch parameters.
"""
import importlib

__all__ = ["ptap", "problems", "autotune", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
