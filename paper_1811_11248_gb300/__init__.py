"""GB300-native hierarchical solver with deferred compression.

The solver itself is the C-ABI library built from ``csrc/`` (CUDA for
sm_103a plus host C++); ``hsolve`` is its thin ctypes binding.  ``inputs``
holds the seeded synthetic problems.  Submodules load lazily so that the
input generator can be used without the CUDA library.
"""
__all__ = ["inputs", "hsolve"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
