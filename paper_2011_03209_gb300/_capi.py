"""ctypes declarations of the C ABI in include/mapper.h.

Loading fails loudly when the compiled library is absent: there is no CPU
fallback for any step of the mapper path.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmapper_gb300.so")
# the checked build (device-side index checks); MAPPER_CHECKED=1 loads it instead
CHECKED_LIB_PATH = os.path.join(_HERE, "_build", "libmapper_gb300_checked.so")

MAPPER_OK = 0
MAPPER_EINVAL = -1
MAPPER_ENOMEM = -2
MAPPER_ECUDA = -3
MAPPER_ETIMEOUT = -4
MAPPER_ENONFINITE = -5
MAPPER_EINTERNAL = -6
MAPPER_ENOTIMPL = -7
MAPPER_ECANCELED = -8

LENS_L2, LENS_COORD, LENS_PCA, LENS_ECC, LENS_LINF, LENS_DENSITY, LENS_ECC_INF = 0, 1, 2, 3, 4, 5, 6
COVER_UNIFORM, COVER_BALANCED = 0, 1
FP32, BF16, BF16X1, FP8 = 0, 1, 2, 3

# every symbol include/mapper.h declares
EXPORTS = (
    "mapper_create", "mapper_destroy", "mapper_set_stream", "mapper_set_timing", "mapper_set_pass1_tile_n",
    "mapper_set_cross_screen", "mapper_selftest_wait", "mapper_set_knn_screen", "mapper_knn_info", "mapper_set_band_queue_cap",
    "mapper_set_pass1_screen", "mapper_selftest_mma_error", "mapper_single_linkage", "mapper_forest_sizes",
    "mapper_forest_copy", "mapper_forest_cut",
    "mapper_cover_subset", "mapper_nerve_from_nodes", "mapper_cover_balanced", "mapper_knn_distance",
    "mapper_lens", "mapper_lens_ex", "mapper_cover", "mapper_cover_sizes", "mapper_cover_copy",
    "mapper_cluster", "mapper_clusters_copy", "mapper_nerve", "mapper_graph",
    "mapper_graph_sizes", "mapper_graph_copy", "mapper_graph_lens", "mapper_graph_cover",
    "mapper_graph_clusters", "mapper_stats_get", "mapper_free", "mapper_strerror",
    "mapper_last_error", "mapper_abi_version", "mapper_dbscan_noalloc", "mapper_graph_footprint",
    "mapper_server_create", "mapper_server_destroy", "mapper_server_add_dataset", "mapper_server_submit",
    "mapper_server_wait", "mapper_server_load", "mapper_graph_sweep",
)

NOALLOC_MAX_POINTS = 8192
NOALLOC_MAX_DIM = 256


class MapperParams(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int32),
        ("lens_kind", ctypes.c_int32 * 2),
        ("lens_arg", ctypes.c_int32 * 2),
        ("n_intervals", ctypes.c_int32 * 2),
        ("overlap", ctypes.c_double * 2),
        ("eps", ctypes.c_double),
        ("min_pts", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("cover_kind", ctypes.c_int32),
        ("lens_param", ctypes.c_double * 2),
    ]


class MapperStats(ctypes.Structure):
    _fields_ = [
        ("n_points", ctypes.c_int64),
        ("n_elements", ctypes.c_int64),
        ("n_members", ctypes.c_int64),
        ("sum_ni2", ctypes.c_double),
        ("tile_pairs", ctypes.c_int64),
        ("tile_pairs_out", ctypes.c_int64),
        ("tile_pairs_in", ctypes.c_int64),
        ("pairs_screened", ctypes.c_int64),
        ("band_pairs", ctypes.c_int64),
        ("near_ties", ctypes.c_int64),
        ("n_core", ctypes.c_int64),
        ("n_nodes", ctypes.c_int64),
        ("n_edges", ctypes.c_int64),
        ("n_launches", ctypes.c_int64),
        ("ms_lens", ctypes.c_double),
        ("ms_cover", ctypes.c_double),
        ("ms_cluster", ctypes.c_double),
        ("ms_nerve", ctypes.c_double),
        ("ms_total", ctypes.c_double),
        ("ms_pass", ctypes.c_double * 3),
        ("ms_tiles", ctypes.c_double),
        ("tile_pairs_tc", ctypes.c_int64),
        ("tile_pairs_simt", ctypes.c_int64),
        ("union_skipped", ctypes.c_int64),
        ("n_groups", ctypes.c_int64),
        ("n_rows", ctypes.c_int64),
        ("count_kernel_pairs", ctypes.c_int64),
        ("ms_count_kernel", ctypes.c_double),
        ("union_pairs", ctypes.c_int64),
        ("fp64_pairs", ctypes.c_int64),
        ("pass1_tile_n", ctypes.c_int64),
        ("tile_pairs_cross", ctypes.c_int64),
        ("tile_pairs_screen1", ctypes.c_int64),
        ("tile_pairs_redo", ctypes.c_int64),
        ("redo_blocks", ctypes.c_int64),
        ("redo_parts", ctypes.c_int64),
        ("pass1_phases", ctypes.c_int64),
        ("pass1_sample_deferred", ctypes.c_double),
        ("tile_pairs_direct", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        out = {name: getattr(self, name) for name, _ in self._fields_}
        out["ms_pass"] = list(self.ms_pass)
        return out


class RequestInfo(ctypes.Structure):
    _fields_ = [
        ("queue_s", ctypes.c_double),
        ("run_s", ctypes.c_double),
        ("latency_s", ctypes.c_double),
        ("footprint", ctypes.c_size_t),
        ("status", ctypes.c_int32),
    ]


class MapperError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status}: {message}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load the library (once). Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or (CHECKED_LIB_PATH if os.environ.get("MAPPER_CHECKED") == "1" else LIB_PATH)
        if not os.path.exists(p):
            raise RuntimeError(
                f"CUDA library {p} is missing: build it first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(p)
        P = ctypes.c_void_p
        PP = ctypes.POINTER(ctypes.c_void_p)
        i32, i64, f64, sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
        sig = {
            "mapper_create": (ctypes.c_int, [PP, ctypes.c_int, sz, P]),
            "mapper_destroy": (None, [P]),
            "mapper_set_stream": (ctypes.c_int, [P, P]),
            "mapper_set_timing": (ctypes.c_int, [P, ctypes.c_int]),
            "mapper_set_pass1_tile_n": (ctypes.c_int, [P, ctypes.c_int]),
            "mapper_set_cross_screen": (ctypes.c_int, [P, ctypes.c_int]),
            "mapper_selftest_wait": (ctypes.c_int, [P]),
            "mapper_set_knn_screen": (ctypes.c_int, [P, ctypes.c_int]),
            "mapper_knn_info": (ctypes.c_int, [P, P]),
            "mapper_set_band_queue_cap": (ctypes.c_int, [P, i64]),
            "mapper_set_pass1_screen": (ctypes.c_int, [P, ctypes.c_int]),
            "mapper_single_linkage": (ctypes.c_int, [P, P, i64, i32, i64, P, f64, ctypes.POINTER(P)]),
            "mapper_forest_sizes": (ctypes.c_int, [P, ctypes.POINTER(i64)]),
            "mapper_forest_copy": (ctypes.c_int, [P, P, P, P, P, ctypes.c_int]),
            "mapper_forest_cut": (ctypes.c_int, [P, P, f64, ctypes.POINTER(P)]),
            "mapper_selftest_mma_error": (ctypes.c_int, [P, i32, i32, i32, ctypes.c_uint64, ctypes.POINTER(f64),
                                                         ctypes.POINTER(f64)]),
            "mapper_cover_subset": (ctypes.c_int, [P, P, P, ctypes.c_int32, ctypes.POINTER(P)]),
            "mapper_nerve_from_nodes": (ctypes.c_int, [P, ctypes.c_int64, ctypes.c_int64, P, P, P,
                                                       ctypes.POINTER(P)]),
            "mapper_lens": (ctypes.c_int, [P, P, i64, i32, i64, i32, P, P, P, P]),
            "mapper_lens_ex": (ctypes.c_int, [P, P, i64, i32, i64, i32, P, P, P, i32, P, P]),
            "mapper_cover": (ctypes.c_int, [P, P, i64, i32, P, P, PP]),
            "mapper_cover_balanced": (ctypes.c_int, [P, P, i64, i32, P, P, PP]),
            "mapper_knn_distance": (ctypes.c_int, [P, P, i64, i32, i64, P, i64, i32, P]),
            "mapper_cover_sizes": (ctypes.c_int, [P, P, P]),
            "mapper_cover_copy": (ctypes.c_int, [P, P, P, ctypes.c_int]),
            "mapper_cluster": (ctypes.c_int, [P, P, i64, i32, i64, P, f64, i32, i32, PP]),
            "mapper_clusters_copy": (ctypes.c_int, [P, P, P, ctypes.c_int]),
            "mapper_nerve": (ctypes.c_int, [P, P, PP]),
            "mapper_graph": (ctypes.c_int, [P, P, i64, i32, i64, ctypes.POINTER(MapperParams), PP]),
            "mapper_graph_sizes": (ctypes.c_int, [P, P, P, P]),
            "mapper_graph_copy": (ctypes.c_int, [P, P, P, P, P, ctypes.c_int]),
            "mapper_graph_lens": (ctypes.c_int, [P, P, P, P, ctypes.c_int]),
            "mapper_graph_cover": (P, [P]),
            "mapper_graph_clusters": (P, [P]),
            "mapper_stats_get": (ctypes.c_int, [P, ctypes.POINTER(MapperStats)]),
            "mapper_free": (None, [P]),
            "mapper_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "mapper_last_error": (ctypes.c_char_p, []),
            "mapper_abi_version": (ctypes.c_int, []),
            "mapper_dbscan_noalloc": (ctypes.c_int, [P, i64, i32, i64, f64, i32, P, P, P]),
            "mapper_graph_footprint": (ctypes.c_int, [i64, i32, ctypes.POINTER(MapperParams), P]),
            "mapper_graph_sweep": (ctypes.c_int, [P, P, i64, i32, i64, ctypes.POINTER(MapperParams), i32, P, P,
                                                  P]),
            "mapper_server_create": (ctypes.c_int, [PP, ctypes.c_int, ctypes.c_int, sz]),
            "mapper_server_destroy": (None, [P]),
            "mapper_server_add_dataset": (ctypes.c_int, [P, P, i64, i32, i64, P]),
            "mapper_server_submit": (ctypes.c_int, [P, i32, ctypes.POINTER(MapperParams), P]),
            "mapper_server_wait": (ctypes.c_int, [P, i64, f64, PP, ctypes.POINTER(RequestInfo)]),
            "mapper_server_load": (ctypes.c_int, [P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(status: int, where: str) -> None:
    if status != MAPPER_OK:
        lib = load()
        raise MapperError(status, where, lib.mapper_last_error().decode(errors="replace"))
