"""ctypes declarations of the C ABI in ``include/exactmap.h``.

Argument marshalling only: every step of the mapping runs in the CUDA
library.  Loading fails loudly when ``libexactmap.so`` has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libexactmap.so")

EM_OK, EM_EINVAL, EM_ENOMEM, EM_ECUDA, EM_ECAPACITY, EM_ENOTCONV, EM_ETIMEOUT = range(7)
STATUS_NAMES = {0: "EM_OK", 1: "EM_EINVAL", 2: "EM_ENOMEM", 3: "EM_ECUDA", 4: "EM_ECAPACITY",
                5: "EM_ENOTCONV", 6: "EM_ETIMEOUT"}


class EmParams(C.Structure):
    _fields_ = [("r_part", C.c_double), ("r_leaf", C.c_double), ("theta", C.c_double),
                ("h_fact", C.c_double), ("h_tol", C.c_double), ("max_newton", C.c_int),
                ("precision", C.c_int), ("fp64_threshold", C.c_double), ("knn_k", C.c_int),
                ("leaf_max", C.c_int), ("block_pairs", C.c_int), ("h0_above", C.c_int),
                ("fp32_err_ulps", C.c_int), ("fp32_variant", C.c_int), ("reserved", C.c_int * 2)]


class EmSnapshot(C.Structure):
    _fields_ = [("n", C.c_int64), ("d_x", C.c_void_p), ("d_y", C.c_void_p), ("d_z", C.c_void_p),
                ("d_m", C.c_void_p), ("d_h", C.c_void_p), ("ngen", C.c_int64), ("d_gx", C.c_void_p),
                ("d_gy", C.c_void_p), ("d_gz", C.c_void_p), ("box", C.c_double * 6), ("nsrc", C.c_int),
                ("h_src", C.c_void_p), ("d_f_cell", C.c_void_p), ("d_rho", C.c_void_p), ("d_f", C.c_void_p),
                ("npseudo", C.c_int64), ("npairs", C.c_int64), ("nfp64", C.c_int64), ("status", C.c_int)]


P = C.c_void_p
PP = C.POINTER(C.c_void_p)
I64 = C.c_int64
I32 = C.c_int
D = C.c_double
PI64 = C.POINTER(C.c_int64)
PI32 = C.POINTER(C.c_int32)
PPAR = C.POINTER(EmParams)

# name -> (restype, argtypes); every symbol declared in include/exactmap.h
SIGNATURES = {
    "em_params_default": (None, [PPAR]),
    "em_ctx_create": (I32, [PP, I32, P]),
    "em_ctx_destroy": (I32, [P]),
    "em_ctx_sync": (I32, [P]),
    "em_last_error": (C.c_char_p, []),
    "em_ctx_launch_count": (I64, [P]),
    "em_ctx_set_timing": (I32, [P, I32]),
    "em_ctx_map_times": (I32, [P, P, P]),
    "em_measure_peaks": (I32, [P, P]),
    "build_tree": (I32, [P, I64, P, P, P, P, P, I32, PP]),
    "tree_info": (I32, [P, PI64, PI64, PI32]),
    "tree_get": (I32, [P, P] + [P] * 11),
    "tree_destroy": (I32, [P]),
    "make_pseudo_particles": (I32, [P, P, P, I32, P, PPAR, PP]),
    "make_pseudo_particles_forced": (I32, [P, P, P, I32, P, PPAR, P, PP]),
    "refine_check": (I32, [P, P, P, P, D, I32, P, PI64, PI64]),
    "pseudo_info": (I32, [P, PI64, PI64]),
    "pseudo_get": (I32, [P, P] + [P] * 9),
    "pseudo_destroy": (I32, [P]),
    "build_voronoi": (I32, [P, I64, P, P, P, P, PPAR, PP]),
    "build_voronoi_cells": (I32, [P, I64, P, P, P, P, PPAR, I64, I64, PP]),
    "voronoi_from_cells": (I32, [P, I64, I64, I64, P, P, P, P, P, P, P, PP]),
    "voronoi_info": (I32, [P, PI64, PI64, PI64]),
    "voronoi_centroids": (I32, [P, P, P, P, P]),
    "lloyd": (I32, [P, I64, P, P, P, P, I32, PPAR]),
    "map_batch": (I32, [I32, I32, C.POINTER(EmSnapshot), PPAR, I32, I32, PI32, P, PI64]),
    "map_batch_create": (I32, [I32, PPAR, I32, PP]),
    "map_batch_add": (I32, [P, C.POINTER(EmSnapshot), PI32]),
    "map_batch_run": (I32, [P, I32, PI32, P, PI64]),
    "map_batch_get": (I32, [P, I32, C.POINTER(EmSnapshot)]),
    "map_batch_destroy": (I32, [P]),
    "voronoi_get": (I32, [P, P] + [P] * 6),
    "voronoi_destroy": (I32, [P]),
    "find_pairs": (I32, [P, I64, P, P, P, P, P, PP, PI64]),
    "find_pairs_plan": (I32, [P, I64, P, P, P, P, P, I64, P, PI64, PI64]),
    "find_pairs_cells": (I32, [P, I64, P, P, P, P, P, I64, I64, I64, PP, PI64]),
    "map_back_sums": (I32, [P, P, P, P, P, P]),
    "inherit": (I32, [P, P, P, P, P]),
    "pairs_from_list": (I32, [P, I64, P, P, I64, P, PP]),
    "pairs_info": (I32, [P, PI64, PI64, PI64]),
    "pairs_get": (I32, [P, P, P, P, P, P]),
    "pairs_destroy": (I32, [P]),
    "map_exact": (I32, [P, P, P, P, P, P, P, P, PPAR, P, P, P, PI64]),
    "map_exact_noalloc": (I32, [P, P, P, P, P, P, P, P, PPAR, P, P, P, PI64]),
    "map_autotune": (I32, [P, P, P, P, P, P, P, PPAR, PI32, P]),
    "map_back": (I32, [P, P, P, P, P, P, P, P]),
}

_lib = None


class NativeError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn} failed with {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    """The loaded library; raises if it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'` "
                              "(the mapping has no CPU path)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(fn_name: str, status: int, allow=(EM_OK,)):
    if status not in allow:
        raise NativeError(fn_name, status, lib().em_last_error().decode(errors="replace"))
    return status


def call(name: str, *args, allow=(EM_OK,)):
    return check(name, getattr(lib(), name)(*args), allow)
