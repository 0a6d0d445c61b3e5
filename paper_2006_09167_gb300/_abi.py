"""ctypes declarations of the C ABI in include/nb.h (argument marshalling only).

The shared library is loaded from this package directory.  There is no
fallback: if libnb.so is missing or cannot be loaded, importing this module
raises, so nothing can silently run on another code path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnb.so")

NB_OK = 0
NB_ERR_INVALID_ARG = 1
NB_ERR_BOX_TOO_SMALL = 2
NB_ERR_NOT_READY = 3
NB_ERR_CAPACITY = 4
NB_ERR_CUDA = 5
NB_ERR_TIMEOUT = 6
NB_ERR_NONFINITE = 7

NB_COULOMB_RF = 0
NB_COULOMB_EWALD = 1
NB_COULOMB_NONE = 2
NB_ENERGY = 1
NB_VIRIAL = 2
NB_LIST_OUTER = 0
NB_LIST_INNER = 1

# every entry point declared in include/nb.h
EXPORTED = [
    "nb_create", "nb_destroy", "nb_set_charges", "nb_set_lj", "nb_grid_sort", "nb_pairlist_build",
    "nb_prune_rolling", "nb_forces", "nb_forces_vjp", "nb_batch_create", "nb_batch_destroy",
    "nb_forces_batched", "nb_count_pairs", "nb_debug_export_pairs", "nb_debug_layout",
    "nb_get_stats", "nb_get_error", "nb_status_str", "nb_trace_enable", "nb_trace_read",
    "nb_forces_small_noalloc", "nb_set_split", "nb_pme_create", "nb_pme_destroy", "nb_pme_forces",
    "nb_ewald_corrections", "nb_set_fused_prune", "nb_sorted_export", "nb_forces_sorted", "nb_forces_vjp_dev",
    "nb_set_search_segments",
]
NB_NOALLOC_MAX_ATOMS = 16384
NB_NOALLOC_MAX_TYPES = 8
NB_TRACE_FORCES = 0
NB_TRACE_PRUNE = 1
NB_TRACE_GATHER = 2
NB_TRACE_VJP = 3
NB_TRACE_KINDS = 4


class NbParams(ctypes.Structure):
    _fields_ = [
        ("n_atoms", ctypes.c_int32), ("n_types", ctypes.c_int32), ("coulomb", ctypes.c_int32),
        ("reserved", ctypes.c_int32), ("eps_r", ctypes.c_double), ("eps_rf", ctypes.c_double),
        ("beta", ctypes.c_double), ("rc", ctypes.c_double), ("rlist", ctypes.c_double),
        ("r_in", ctypes.c_double), ("c6_host", ctypes.POINTER(ctypes.c_float)),
        ("c12_host", ctypes.POINTER(ctypes.c_float)),
    ]


class NbPmeParams(ctypes.Structure):
    _fields_ = [
        ("n_atoms", ctypes.c_int32), ("grid", ctypes.c_int32 * 3), ("order", ctypes.c_int32),
        ("reserved", ctypes.c_int32), ("beta", ctypes.c_double), ("eps_r", ctypes.c_double),
    ]


class NbStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "n_atoms", "n_slots", "n_clusters", "n_superclusters", "n_items", "n_outer_j",
        "n_outer_bits", "n_mask_groups", "grid_nx", "grid_ny", "n_launches")]


class NbError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_str(status)} (status {status})")


_lib = None


def load(path: str = LIB_PATH):
    """Load libnb.so (raises OSError if it is missing: build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} is not built; call paper_2006_09167_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    i32p = ctypes.POINTER(ctypes.c_int32)
    f32p = ctypes.POINTER(ctypes.c_float)
    i64p = ctypes.POINTER(ctypes.c_int64)
    st = ctypes.c_int
    lib.nb_create.argtypes = [ctypes.POINTER(NbParams), f32p, i32p, i32p, i32p, ctypes.POINTER(vp)]
    lib.nb_create.restype = st
    lib.nb_destroy.argtypes = [vp]
    lib.nb_destroy.restype = None
    lib.nb_set_charges.argtypes = [vp, vp, vp]
    lib.nb_set_lj.argtypes = [vp, vp, vp, vp]
    lib.nb_grid_sort.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double), vp]
    lib.nb_pairlist_build.argtypes = [vp, ctypes.c_float, vp]
    lib.nb_prune_rolling.argtypes = [vp, ctypes.c_float, ctypes.c_int, ctypes.c_int, vp]
    lib.nb_forces.argtypes = [vp, ctypes.c_uint, vp, vp, vp, vp, vp]
    lib.nb_forces_vjp.argtypes = [vp, vp, vp, ctypes.c_double, vp, vp, vp, vp, vp]
    lib.nb_sorted_export.argtypes = [vp, vp, vp, vp]
    lib.nb_forces_vjp_dev.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.nb_forces_sorted.argtypes = [vp, ctypes.c_uint, vp, vp, vp, vp, vp]
    lib.nb_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp)]
    lib.nb_batch_destroy.argtypes = [vp]
    lib.nb_batch_destroy.restype = None
    lib.nb_forces_batched.argtypes = [vp, ctypes.c_uint, vp, vp, vp, vp, vp]
    lib.nb_count_pairs.argtypes = [vp, ctypes.c_int, i64p, i64p, vp]
    lib.nb_debug_export_pairs.argtypes = [vp, ctypes.c_int, i64p, ctypes.c_size_t,
                                          ctypes.POINTER(ctypes.c_size_t), vp]
    lib.nb_debug_layout.argtypes = [vp, i32p, f32p, f32p, vp]
    lib.nb_get_stats.argtypes = [vp, ctypes.POINTER(NbStats)]
    lib.nb_get_error.argtypes = [vp, vp]
    lib.nb_set_split.argtypes = [vp, ctypes.c_int]
    lib.nb_set_search_segments.argtypes = [vp, ctypes.c_int]
    lib.nb_set_fused_prune.argtypes = [vp, ctypes.c_int]
    lib.nb_trace_enable.argtypes = [vp, ctypes.c_int]
    lib.nb_trace_read.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), i64p]
    lib.nb_forces_small_noalloc.argtypes = [ctypes.POINTER(NbParams), vp, vp, vp, vp, vp,
                                            ctypes.POINTER(ctypes.c_double), ctypes.c_uint, vp, vp, vp, vp]
    lib.nb_pme_create.argtypes = [ctypes.POINTER(NbPmeParams), ctypes.POINTER(vp)]
    lib.nb_pme_destroy.argtypes = [vp]
    lib.nb_pme_destroy.restype = None
    lib.nb_pme_forces.argtypes = [vp, ctypes.c_uint, vp, vp, ctypes.POINTER(ctypes.c_double), vp, vp, vp, vp]
    lib.nb_ewald_corrections.argtypes = [vp, ctypes.c_uint, vp, vp, vp, vp, vp]
    lib.nb_status_str.argtypes = [ctypes.c_int]
    lib.nb_status_str.restype = ctypes.c_char_p
    for name in EXPORTED:
        fn = getattr(lib, name)
        if name not in ("nb_destroy", "nb_batch_destroy", "nb_pme_destroy", "nb_status_str") and fn.restype is not st:
            fn.restype = st
    _lib = lib
    return lib


def status_str(s: int) -> str:
    try:
        return load().nb_status_str(int(s)).decode()
    except OSError:
        return f"status {s}"


def check(status: int, where: str) -> None:
    if status != NB_OK:
        raise NbError(status, where)
