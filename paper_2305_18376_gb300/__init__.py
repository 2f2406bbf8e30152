"""GB300-native Dash: dual-way streaming PARAFAC2 updates (Jang, Jang and
Kang, KDD'23) as hand-written CUDA for sm_103a behind a C ABI
(include/dash.h).  This package holds the CUDA sources (csrc/), the in-tree
build (build.py) and a thin ctypes binding (_native.py)."""
from ._native import DashError, DashModel, LIB_PATH, load  # noqa: F401

__all__ = ["DashModel", "DashError", "load", "LIB_PATH"]
