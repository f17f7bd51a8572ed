"""GB300 U-HNSW query path (arxiv 2605.02030): C-ABI library libuhnsw.so
(include/uhnsw.h) with sm_103a CUDA kernels, and its Python binding."""
from ._build import build  # noqa: F401


def __getattr__(name):
    # the binding is imported lazily so that `inputs` can be used without torch
    if name in ("Index", "build_graph", "load_library", "UHNSWError", "library_path"):
        from . import uhnsw
        return getattr(uhnsw, name)
    raise AttributeError(name)
