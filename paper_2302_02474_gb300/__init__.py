"""GB300-native TILD timestep (MATILDA.FT, arXiv 2302.02474).

The compute path is a CUDA library (``_lib/libtild.so``, built from
``csrc/`` for sm_103a) behind the C ABI in ``include/tild.h``; ``binding``
marshals arguments to it with ctypes. ``inputs`` builds seeded synthetic
systems. Importing the package does not load the library; the first use
of ``binding`` does, and fails loudly if it has not been built.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "binding"]


def __getattr__(name):
    if name == "binding":
        import importlib

        return importlib.import_module(__name__ + ".binding")
    raise AttributeError(name)
