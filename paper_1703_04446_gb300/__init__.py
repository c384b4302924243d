"""GB300-native Lagrangian Gauss-Newton-Krylov hot path (arXiv 1703.04446).

``lgnk``   ctypes binding of the C ABI in include/lgnk.h (CUDA library liblgnk.so)
``synth``  seeded synthetic inputs shaped like the paper's problems
``build``  in-tree nvcc build of liblgnk.so for sm_103a

The binding is imported lazily so that ``synth`` works without torch or the
built library.
"""

__all__ = ["lgnk", "synth", "build"]


def __getattr__(name):
    if name in ("lgnk", "synth", "build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
