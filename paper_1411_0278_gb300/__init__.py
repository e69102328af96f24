"""GB300-native Galerkin boundary-integral solver for N active spheres.

The method (Singh, Ghose & Adhikari, arXiv:1411.0278) runs in libgbi, a C-ABI
CUDA library for sm_103a (``include/gbi.h``); this package holds its sources
(``csrc/``), the build step (``build.py``, ``gen_tables.py``) and a thin ctypes
binding (``_native``).  The library is loaded on first use and its absence is an
error: there is no CPU path.
"""
from ._native import (GBI_ERR_ARG, GBI_ERR_CUDA, GBI_ERR_NOMEM, GBI_ERR_NOT_CONVERGED, GBI_ERR_OVERLAP,
                      GBI_ERR_TIMEOUT, GBI_OK, SET_ALL, SET_H, SET_L, Context, GbiError, component_scales, d,
                      gbi_info, gbi_params, h, lib, params, self_scalars, solve_static, status_string)

__all__ = ["Context", "GbiError", "params", "solve_static", "gbi_params", "gbi_info", "h", "d", "component_scales",
           "self_scalars", "status_string", "lib", "SET_ALL", "SET_L", "SET_H", "GBI_OK", "GBI_ERR_ARG",
           "GBI_ERR_OVERLAP", "GBI_ERR_NOT_CONVERGED", "GBI_ERR_TIMEOUT", "GBI_ERR_CUDA", "GBI_ERR_NOMEM"]
