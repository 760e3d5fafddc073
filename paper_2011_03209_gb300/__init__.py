"""GB300-native mapper graph ("Mapper Interactive", arXiv 2011.03209, §3).

Thin Python binding over the C ABI of libmapper_gb300.so (include/mapper.h).
The functions carry the C names: `mapper_lens`, `mapper_cover`,
`mapper_cluster`, `mapper_nerve` and the fused `mapper_graph`. They only
marshal arguments: every step runs in the library's CUDA kernels. PyTorch
supplies device memory and streams.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _capi
from ._capi import (BF16, BF16X1, COVER_BALANCED, COVER_UNIFORM, FP8, FP32, LENS_COORD, LENS_DENSITY, LENS_ECC,
                    LENS_ECC_INF, LENS_L2, LENS_LINF, LENS_PCA,
                    MapperError, MapperParams)

__all__ = [
    "Context", "Cover", "Clusters", "Graph", "MapperError", "mapper_lens", "mapper_cover",
    "mapper_cluster", "mapper_nerve", "mapper_graph", "params", "LENS_L2", "LENS_COORD",
    "LENS_PCA", "LENS_ECC", "LENS_LINF", "LENS_DENSITY", "LENS_ECC_INF", "COVER_UNIFORM", "COVER_BALANCED", "FP32", "BF16", "BF16X1", "FP8", "mapper_dbscan_noalloc", "Server", "graph_footprint",
    "mapper_graph_sweep", "mapper_cover_subset", "mapper_nerve_from_nodes", "mapper_knn_distance",
    "mapper_single_linkage", "Forest",
]


def _torch():
    import torch
    return torch


def _vp(x) -> ctypes.c_void_p:
    return ctypes.c_void_p(int(x))


class Context:
    """A library context bound to one CUDA device and stream."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, stream=None):
        self._lib = _capi.load()
        h = ctypes.c_void_p()
        s = None if stream is None else _vp(stream.cuda_stream)
        _capi.check(self._lib.mapper_create(ctypes.byref(h), int(device), int(hbm_budget), s),
                    "mapper_create")
        self.h = h
        self.device = int(device)
        self._stream = stream

    def set_stream(self, stream) -> None:
        _capi.check(self._lib.mapper_set_stream(self.h, _vp(stream.cuda_stream)), "mapper_set_stream")
        self._stream = stream

    def set_timing(self, on: bool) -> None:
        _capi.check(self._lib.mapper_set_timing(self.h, int(bool(on))), "mapper_set_timing")

    def set_pass1_tile_n(self, tile_n: int) -> None:
        """0: autotuned (default); 128 or 256: fixed pass-1 product shape."""
        _capi.check(self._lib.mapper_set_pass1_tile_n(self.h, int(tile_n)), "mapper_set_pass1_tile_n")

    def set_knn_screen(self, mode: int) -> None:
        """k-distance screen: 0 tensor cores (default), 1 tensor cores, 2 CUDA
        cores, 3 tensor cores without the sampled threshold."""
        _capi.check(self._lib.mapper_set_knn_screen(self.h, int(mode)), "mapper_set_knn_screen")

    def knn_info(self) -> dict:
        """The path of the last mapper_knn_distance call: path (0 CUDA cores,
        1 tensor-core lists, 2 sampled threshold), queries over capacity, the
        capacity per query, the sample's tile stride, the keys below the
        thresholds (all queries, and the most of one query) and the merge's
        FP32 and FP64 candidates."""
        info = (ctypes.c_int64 * 8)()
        _capi.check(self._lib.mapper_knn_info(self.h, info), "mapper_knn_info")
        return {"path": int(info[0]), "over_capacity": int(info[1]), "capacity": int(info[2]),
                "sample_stride": int(info[3]), "keys": int(info[4]), "max_keys": int(info[5]),
                "fp32_candidates": int(info[6]), "fp64_candidates": int(info[7])}

    def set_cross_screen(self, mode: int) -> None:
        """Mixed tile pairs across two segments: 0 auto (default), 1 tensor
        cores, 2 CUDA cores."""
        _capi.check(self._lib.mapper_set_cross_screen(self.h, int(mode)), "mapper_set_cross_screen")

    def set_pass1_screen(self, mode: int) -> None:
        """MAPPER_BF16 count pass: 0 default, 1 two phases (one product, then
        three for the tile pairs with a band pair), 2 three products."""
        _capi.check(self._lib.mapper_set_pass1_screen(self.h, int(mode)), "mapper_set_pass1_screen")

    def selftest_mma_error(self, dp: int, products: int, seed: int = 1, fmt: int = 0):
        """(observed, modelled) accumulation error of the tensor-core screen's
        products on random BF16 (fmt 0) or FP8 E4M3 (fmt 1) rows, both
        relative to the magnitude sum."""
        o, m = ctypes.c_double(), ctypes.c_double()
        _capi.check(self._lib.mapper_selftest_mma_error(self.h, int(dp), int(products), int(fmt), int(seed),
                                                        ctypes.byref(o), ctypes.byref(m)),
                    "mapper_selftest_mma_error")
        return o.value, m.value

    def set_band_queue_cap(self, entries: int) -> None:
        """Band-queue capacity in pairs (0: sized from the tile pairs, the
        default); band pairs past it are decided inside the screen kernel."""
        _capi.check(self._lib.mapper_set_band_queue_cap(self.h, int(entries)), "mapper_set_band_queue_cap")

    def close(self) -> None:
        if getattr(self, "h", None) is not None and self.h.value:
            self._lib.mapper_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Handle:
    def __init__(self, lib, h, owner=None):
        self._lib = lib
        self.h = h
        self._owner = owner           # views keep their graph alive

    def _free(self):
        if self._owner is None and getattr(self, "h", None) is not None and self.h.value:
            self._lib.mapper_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self._free()
        except Exception:
            pass

    def stats(self) -> dict:
        st = _capi.MapperStats()
        _capi.check(self._lib.mapper_stats_get(self.h, ctypes.byref(st)), "mapper_stats_get")
        return st.as_dict()


class Cover(_Handle):
    def sizes(self):
        e, m = ctypes.c_int64(), ctypes.c_int64()
        _capi.check(self._lib.mapper_cover_sizes(self.h, ctypes.byref(e), ctypes.byref(m)),
                    "mapper_cover_sizes")
        return e.value, m.value

    def numpy(self):
        E, M = self.sizes()
        offs = np.empty(E + 1, dtype=np.int64)
        pts = np.empty(max(M, 1), dtype=np.int32)
        _capi.check(self._lib.mapper_cover_copy(self.h, _vp(offs.ctypes.data), _vp(pts.ctypes.data), 0),
                    "mapper_cover_copy")
        return offs, pts[:M]


class Clusters(_Handle):
    def numpy(self, n_members: int):
        lab = np.empty(max(n_members, 1), dtype=np.int64)
        core = np.empty(max(n_members, 1), dtype=np.uint8)
        _capi.check(self._lib.mapper_clusters_copy(self.h, _vp(lab.ctypes.data), _vp(core.ctypes.data), 0),
                    "mapper_clusters_copy")
        return lab[:n_members], core[:n_members].astype(bool)


class Forest(_Handle):
    """Single-linkage forest: the minimum spanning forests of the elements'
    eps-graphs (mapper_single_linkage)."""

    def size(self) -> int:
        k = ctypes.c_int64()
        _capi.check(self._lib.mapper_forest_sizes(self.h, ctypes.byref(k)), "mapper_forest_sizes")
        return k.value

    def numpy(self) -> dict:
        """Edges sorted by (elem, d2, u, v): elem, u < v (points) and d2."""
        k = self.size()
        elem = np.empty(max(k, 1), dtype=np.int32)
        u = np.empty(max(k, 1), dtype=np.int32)
        v = np.empty(max(k, 1), dtype=np.int32)
        d2 = np.empty(max(k, 1), dtype=np.float64)
        _capi.check(self._lib.mapper_forest_copy(self.h, _vp(elem.ctypes.data), _vp(u.ctypes.data),
                                                 _vp(v.ctypes.data), _vp(d2.ctypes.data), 0), "mapper_forest_copy")
        elem, u, v, d2 = elem[:k], u[:k], v[:k], d2[:k]
        order = np.lexsort((v, u, d2, elem))
        return dict(elem=elem[order], u=u[order], v=v[order], d2=d2[order])

    def cut(self, ctx: "Context", h: float) -> Clusters:
        out = ctypes.c_void_p()
        _capi.check(self._lib.mapper_forest_cut(ctx.h, self.h, float(h), ctypes.byref(out)), "mapper_forest_cut")
        return Clusters(self._lib, out)


class Graph(_Handle):
    def sizes(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _capi.check(self._lib.mapper_graph_sizes(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
                    "mapper_graph_sizes")
        return a.value, b.value, c.value

    def numpy(self) -> dict:
        N, G, E = self.sizes()
        no = np.empty(N + 1, dtype=np.int64)
        nm = np.empty(max(G, 1), dtype=np.int32)
        ne = np.empty(max(N, 1), dtype=np.int32)
        ed = np.empty(max(2 * E, 2), dtype=np.int32)
        _capi.check(self._lib.mapper_graph_copy(self.h, _vp(no.ctypes.data), _vp(nm.ctypes.data),
                                                _vp(ne.ctypes.data), _vp(ed.ctypes.data), 0),
                    "mapper_graph_copy")
        return dict(node_offsets=no, node_members=nm[:G], node_elem=ne[:N],
                    edges=ed[:2 * E].reshape(E, 2))

    def lens(self, n: int, m: int):
        """(lens n x m float64, pca basis or None)."""
        f = np.empty((n, m), dtype=np.float64)
        npca = ctypes.c_int64()
        _capi.check(self._lib.mapper_graph_lens(self.h, None, None, ctypes.byref(npca), 0),
                    "mapper_graph_lens")
        pca = np.empty(max(npca.value, 1), dtype=np.float64)
        _capi.check(self._lib.mapper_graph_lens(self.h, _vp(f.ctypes.data), _vp(pca.ctypes.data),
                                                ctypes.byref(npca), 0), "mapper_graph_lens")
        return f, (pca[:npca.value] if npca.value else None)

    def cover(self) -> Cover:
        return Cover(self._lib, ctypes.c_void_p(self._lib.mapper_graph_cover(self.h)), owner=self)

    def clusters(self) -> Clusters:
        return Clusters(self._lib, ctypes.c_void_p(self._lib.mapper_graph_clusters(self.h)), owner=self)


def params(lens_kind, lens_arg, n_intervals, overlap, eps, min_pts, precision=FP32,
           cover_kind=COVER_UNIFORM, lens_param=None) -> MapperParams:
    lens_kind, lens_arg = tuple(lens_kind), tuple(lens_arg)
    n_intervals, overlap = tuple(n_intervals), tuple(overlap)
    p = MapperParams()
    p.m = len(lens_kind)
    for j in range(p.m):
        p.lens_kind[j] = int(lens_kind[j])
        p.lens_arg[j] = int(lens_arg[j])
        p.n_intervals[j] = int(n_intervals[j])
        p.overlap[j] = float(overlap[j])
    p.eps = float(eps)
    p.min_pts = int(min_pts)
    p.precision = int(precision)
    p.cover_kind = int(cover_kind)
    if lens_param is not None:
        for j, r in enumerate(tuple(lens_param)):
            p.lens_param[j] = float(r)
    return p


def _x_args(X):
    """(pointer, n, d, ld, keepalive) for a torch tensor (CUDA or CPU) or a
    NumPy array (host)."""
    if isinstance(X, np.ndarray):
        X = np.ascontiguousarray(X, dtype=np.float32)
        return _vp(X.ctypes.data), X.shape[0], X.shape[1], X.shape[1], X
    torch = _torch()
    if X.dtype != torch.float32 or X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be a 2-D float32 tensor with unit column stride")
    return _vp(X.data_ptr()), X.shape[0], X.shape[1], X.stride(0), X


def mapper_lens(ctx: Context, X, kinds, args, lens_param=None, precision: int = BF16):
    """Lens on the device: returns (lens [n, m] float64 CUDA tensor, pca).
    lens_param[j]: the ball radius of a density lens; precision: the screen
    of its neighbour counts."""
    torch = _torch()
    p, n, d, ld, _keep = _x_args(X)
    m = len(kinds)
    out = torch.empty((n, m), dtype=torch.float64, device=f"cuda:{ctx.device}")
    k = (ctypes.c_int32 * m)(*kinds)
    a = (ctypes.c_int32 * m)(*args)
    lp = (ctypes.c_double * m)(*[float(r) for r in lens_param]) if lens_param is not None else None
    npca = d * (1 + max([arg for kind, arg in zip(kinds, args) if kind == LENS_PCA], default=-1))
    pca = np.empty(max(npca, 1), dtype=np.float64)
    _capi.check(ctx._lib.mapper_lens_ex(ctx.h, p, n, d, ld, m, k, a, lp, int(precision), _vp(out.data_ptr()),
                                        _vp(pca.ctypes.data) if npca > d else None), "mapper_lens")
    return out, (pca[:npca] if npca > d else None)


def mapper_cover(ctx: Context, lens, n_intervals, overlap, balanced: bool = False) -> Cover:
    n, m = lens.shape
    ni = (ctypes.c_int32 * m)(*n_intervals)
    ov = (ctypes.c_double * m)(*overlap)
    h = ctypes.c_void_p()
    fn = ctx._lib.mapper_cover_balanced if balanced else ctx._lib.mapper_cover
    _capi.check(fn(ctx.h, _vp(lens.data_ptr()), n, m, ni, ov, ctypes.byref(h)), "mapper_cover")
    return Cover(ctx._lib, h)


def mapper_single_linkage(ctx: Context, X, cover: Cover, eps: float) -> Forest:
    """Minimum spanning forests of the cover elements' eps-graphs (the
    single-linkage dendrograms up to eps)."""
    p, n, d, ld, _keep = _x_args(X)
    h = ctypes.c_void_p()
    _capi.check(ctx._lib.mapper_single_linkage(ctx.h, p, n, d, ld, cover.h, float(eps), ctypes.byref(h)),
                "mapper_single_linkage")
    return Forest(ctx._lib, h)


def mapper_cluster(ctx: Context, X, cover: Cover, eps: float, min_pts: int, precision: int = FP32) -> Clusters:
    p, n, d, ld, _keep = _x_args(X)
    h = ctypes.c_void_p()
    _capi.check(ctx._lib.mapper_cluster(ctx.h, p, n, d, ld, cover.h, float(eps), int(min_pts),
                                        int(precision), ctypes.byref(h)), "mapper_cluster")
    c = Clusters(ctx._lib, h)
    c._cover = cover
    return c


def mapper_nerve(ctx: Context, clusters: Clusters) -> Graph:
    h = ctypes.c_void_p()
    _capi.check(ctx._lib.mapper_nerve(ctx.h, clusters.h, ctypes.byref(h)), "mapper_nerve")
    return Graph(ctx._lib, h)


def mapper_knn_distance(ctx: Context, X, queries, k: int) -> np.ndarray:
    """Distance from each query row to its k-th nearest row of X (the row
    itself first), exact in FP64. X: CUDA tensor."""
    p, n, d, ld, _keep = _x_args(X)
    qs = np.ascontiguousarray(np.asarray(queries, dtype=np.int32))
    out = np.empty(max(qs.size, 1), dtype=np.float64)
    _capi.check(ctx._lib.mapper_knn_distance(ctx.h, p, n, d, ld, _vp(qs.ctypes.data) if qs.size else None,
                                             int(qs.size), int(k), _vp(out.ctypes.data)), "mapper_knn_distance")
    return out[:qs.size]


def mapper_cover_subset(ctx: Context, cover: Cover, elements) -> Cover:
    """A cover of the given elements of `cover` (renumbered in that order)."""
    el = np.ascontiguousarray(np.asarray(elements, dtype=np.int32))
    h = ctypes.c_void_p()
    _capi.check(ctx._lib.mapper_cover_subset(ctx.h, cover.h, _vp(el.ctypes.data) if el.size else None,
                                             int(el.size), ctypes.byref(h)), "mapper_cover_subset")
    return Cover(ctx._lib, h)


def mapper_nerve_from_nodes(ctx: Context, n_points: int, node_offsets, node_members, node_elem) -> Graph:
    """Graph of the given nodes (host arrays) with its nerve edges computed on
    the device."""
    off = np.ascontiguousarray(np.asarray(node_offsets, dtype=np.int64))
    mem = np.ascontiguousarray(np.asarray(node_members, dtype=np.int32))
    elm = np.ascontiguousarray(np.asarray(node_elem, dtype=np.int32))
    N = off.size - 1
    mem_p = mem if mem.size else np.zeros(1, dtype=np.int32)
    elm_p = elm if elm.size else np.zeros(1, dtype=np.int32)
    h = ctypes.c_void_p()
    _capi.check(ctx._lib.mapper_nerve_from_nodes(ctx.h, int(n_points), N, _vp(off.ctypes.data),
                                                 _vp(mem_p.ctypes.data), _vp(elm_p.ctypes.data),
                                                 ctypes.byref(h)), "mapper_nerve_from_nodes")
    return Graph(ctx._lib, h)


def mapper_graph(ctx: Context, X, prm: MapperParams) -> Graph:
    """Fused lens + cover + DBSCAN + nerve. X: CUDA tensor, or a host array
    (copied to the device inside the call)."""
    p, n, d, ld, _keep = _x_args(X)
    h = ctypes.c_void_p()
    _capi.check(ctx._lib.mapper_graph(ctx.h, p, n, d, ld, ctypes.byref(prm), ctypes.byref(h)),
                "mapper_graph")
    return Graph(ctx._lib, h)


def mapper_dbscan_noalloc(X, eps: float, min_pts: int, label=None, core=None, stream=None):
    """DBSCAN of the rows of one CUDA tensor X (n <= 8192, d <= 256) through
    the allocation-free entry point: the library allocates no device memory
    for it (its scratch is a fixed array inside the library). `label` (int64)
    and `core` (uint8) are caller-owned CUDA tensors of n entries, created
    here when not given. Returns (label, core)."""
    torch = _torch()
    p, n, d, ld, _keep = _x_args(X)
    if label is None:
        label = torch.empty(n, dtype=torch.int64, device=X.device)
    if core is None:
        core = torch.empty(n, dtype=torch.uint8, device=X.device)
    s = torch.cuda.current_stream(X.device) if stream is None else stream
    lib = _capi.load()
    _capi.check(lib.mapper_dbscan_noalloc(p, n, d, ld, float(eps), int(min_pts), _vp(label.data_ptr()),
                                          _vp(core.data_ptr()), _vp(s.cuda_stream)),
                "mapper_dbscan_noalloc")
    return label, core


def graph_footprint(n: int, d: int, prm: MapperParams) -> int:
    """Estimated peak device bytes of one mapper_graph call (admission control)."""
    out = ctypes.c_size_t()
    lib = _capi.load()
    _capi.check(lib.mapper_graph_footprint(int(n), int(d), ctypes.byref(prm), ctypes.byref(out)),
                "mapper_graph_footprint")
    return out.value


class Server:
    """Request server over device-resident datasets: requests start as soon as
    a worker slot is free and their footprint fits in the budget; running
    requests overlap on the device (see mapper_server_* in include/mapper.h)."""

    def __init__(self, device: int = 0, n_slots: int = 4, hbm_budget: int = 0):
        self._lib = _capi.load()
        h = ctypes.c_void_p()
        _capi.check(self._lib.mapper_server_create(ctypes.byref(h), int(device), int(n_slots), int(hbm_budget)),
                    "mapper_server_create")
        self.h = h
        self._keep = []

    def add_dataset(self, X) -> int:
        p, n, d, ld, keep = _x_args(X)
        self._keep.append(keep)
        out = ctypes.c_int32()
        _capi.check(self._lib.mapper_server_add_dataset(self.h, p, n, d, ld, ctypes.byref(out)),
                    "mapper_server_add_dataset")
        return out.value

    def submit(self, dataset: int, prm: MapperParams) -> int:
        out = ctypes.c_int64()
        _capi.check(self._lib.mapper_server_submit(self.h, int(dataset), ctypes.byref(prm), ctypes.byref(out)),
                    "mapper_server_submit")
        return out.value

    def wait(self, request: int, timeout: float = -1.0):
        """(Graph, info dict) of a finished request."""
        g = ctypes.c_void_p()
        info = _capi.RequestInfo()
        _capi.check(self._lib.mapper_server_wait(self.h, int(request), float(timeout), ctypes.byref(g),
                                                 ctypes.byref(info)), "mapper_server_wait")
        return Graph(self._lib, g), {k: getattr(info, k) for k, _ in info._fields_}

    def load(self):
        r, q, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _capi.check(self._lib.mapper_server_load(self.h, ctypes.byref(r), ctypes.byref(q), ctypes.byref(b)),
                    "mapper_server_load")
        return r.value, q.value, b.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._lib.mapper_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mapper_graph_sweep(ctx: Context, X, prm: MapperParams, eps, overlap):
    """Graphs for the radii eps[i] with overlaps overlap[i] (all filter
    dimensions), sharing the lens, and the cover and tile layout of each
    distinct overlap. Returns a list of Graph."""
    p, n, d, ld, _keep = _x_args(X)
    k = len(eps)
    if len(overlap) != k:
        raise ValueError("eps and overlap differ in length")
    e = (ctypes.c_double * k)(*[float(x) for x in eps])
    o = (ctypes.c_double * k)(*[float(x) for x in overlap])
    hs = (ctypes.c_void_p * k)()
    _capi.check(ctx._lib.mapper_graph_sweep(ctx.h, p, n, d, ld, ctypes.byref(prm), k, e, o, hs),
                "mapper_graph_sweep")
    return [Graph(ctx._lib, ctypes.c_void_p(h)) for h in hs]
