"""GB300-native cell-wise finite element assembly (the par_loop of Firedrake/PyOP2).

The compute path lives in the CUDA library ``libfe`` (``csrc/``, C-ABI in ``include/fe.h``);
``fe`` is its thin ctypes binding.  ``meshgen`` holds the seeded synthetic inputs.
"""
__all__ = ["meshgen", "fe"]


def __getattr__(name):
    if name in ("fe", "meshgen"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
