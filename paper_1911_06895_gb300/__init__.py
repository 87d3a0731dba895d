"""GB300-native delta-stepping single-source shortest paths.

The hot path -- light/heavy split, frontier light relaxation repeated until the
bucket is stable, the heavy pass and the next-bucket search (Fig. 1 of Sridhar
et al. 2019) -- runs in hand-written CUDA kernels for sm_103a inside
``libdsssp.so``, reached through the C ABI of ``include/dsssp.h``. This package
is the thin Python binding of that ABI. The binding module ``dsssp`` is loaded
on first use of any of its names; it raises ImportError when the library has
not been built (there is no fallback path).
"""
import importlib

_SUBMODULES = ("build", "dsssp", "autograd")


def __getattr__(name):
    if name in _SUBMODULES:
        return importlib.import_module(f"{__name__}.{name}")
    if name.startswith("__"):
        raise AttributeError(name)
    binding = importlib.import_module(f"{__name__}.dsssp")
    try:
        return getattr(binding, name)
    except AttributeError:
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}") from None
