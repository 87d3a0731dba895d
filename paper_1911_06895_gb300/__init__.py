"""GB300-native delta-stepping single-source shortest paths.

The hot path -- light/heavy split, frontier light relaxation repeated until the
bucket is stable, the heavy pass and the next-bucket search (Fig. 1 of Sridhar
et al. 2019) -- runs in hand-written CUDA kernels for sm_103a inside
``libdsssp.so``, reached through the C ABI of ``include/dsssp.h``. This package
is the thin Python binding of that ABI.
"""
from .dsssp import *  # noqa: F401,F403
from .dsssp import Graph, DsssError, make_options, check, EXPORTED, LIB_PATH  # noqa: F401
