"""FP64 CPU oracle of the mapper graph ("Mapper Interactive", §3 Background).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline use it; the product path must never import it, and it shares no
code with the CUDA library.

Lens, cover and per-element DBSCAN run in `mapper_oracle.c` (plain C, double
precision, brute force); this module numbers the nodes and builds the nerve:

  * nodes (§3: "clusters induced by points in f^{-1}(V_k) ... as cover
    elements"): every cluster of every cover element, ordered by (element
    index, canonical id); members in ascending point index;
  * edges (§3: "an edge between i, j if U_i and U_j intersect"): {u, v},
    u < v, whenever some point belongs to both; sorted lexicographically.

Parity status: every function here is pinned by tests against something
other than itself (closed forms, hand-derived fixtures, independent
libraries, brute force) -- see tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mapper_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmapper_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        lib.oracle_lens_l2.argtypes = [P, i64, i32, i64, P]
        lib.oracle_lens_ecc2.argtypes = [P, i64, i32, i64, P]
        lib.oracle_lens_coord.argtypes = [P, i64, i32, i64, i32, P]
        lib.oracle_lens_linf.argtypes = [P, i64, i32, i64, P]
        lib.oracle_lens_density.argtypes = [P, i64, i32, i64, f64, P]
        lib.oracle_lens_ecc_inf.argtypes = [P, i64, i32, i64, P]
        lib.oracle_density_at.argtypes = [P, i64, i32, i64, P, i64, f64, P]
        lib.oracle_lens_project.argtypes = [P, i64, i32, i64, P, P, P]
        lib.oracle_pca.argtypes = [P, i64, i32, i64, i32, P, P, P]
        lib.oracle_pca.restype = ctypes.c_int
        lib.oracle_range.argtypes = [P, i64, i32, i32, P, P]
        lib.oracle_interval_bounds.argtypes = [f64, f64, i32, f64, P, P]
        lib.oracle_cover.argtypes = [P, i64, i32, P, P, i32, P, P]
        lib.oracle_balanced_bounds.argtypes = [P, i64, i32, i32, i32, f64, P, P]
        lib.oracle_cover.restype = i64
        lib.oracle_dbscan.argtypes = [P, i64, i32, i64, P, i64, f64, i32, P, P, P, P]
        lib.oracle_dbscan.restype = ctypes.c_int
        lib.oracle_knn_distance.argtypes = [P, i64, i32, i64, P, i64, i32, P]
        lib.oracle_knn_distance.restype = ctypes.c_int
        lib.oracle_msf.argtypes = [P, i64, i32, i64, P, i64, f64, P, P, P]
        lib.oracle_msf.restype = i64
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    assert X.ndim == 2
    return X


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(t: int) -> None:
    _load().oracle_set_num_threads(int(t))


# ------------------------------------------------------------------ lens --

def lens_l2(X) -> np.ndarray:
    X = _f32(X)
    f = np.empty(X.shape[0], dtype=np.float64)
    _load().oracle_lens_l2(_ptr(X), X.shape[0], X.shape[1], X.shape[1], _ptr(f))
    return f


def lens_ecc2(X) -> np.ndarray:
    """Eccentricity with exponent 2 (root mean squared distance to the cloud),
    O(n^2 d): small clouds only."""
    X = _f32(X)
    f = np.empty(X.shape[0], dtype=np.float64)
    _load().oracle_lens_ecc2(_ptr(X), X.shape[0], X.shape[1], X.shape[1], _ptr(f))
    return f


def lens_linf(X) -> np.ndarray:
    """max_k |x_k| per row."""
    X = _f32(X)
    f = np.empty(X.shape[0], dtype=np.float64)
    _load().oracle_lens_linf(_ptr(X), X.shape[0], X.shape[1], X.shape[1], _ptr(f))
    return f


def lens_density(X, r: float) -> np.ndarray:
    """Number of points within distance r of each row (itself included),
    O(n^2 d): small clouds only."""
    X = _f32(X)
    f = np.empty(X.shape[0], dtype=np.float64)
    _load().oracle_lens_density(_ptr(X), X.shape[0], X.shape[1], X.shape[1], float(r), _ptr(f))
    return f


def density_at(X, queries, r: float) -> np.ndarray:
    """The density filter (points within distance r, the point included) at
    the given rows only."""
    X = _f32(X)
    qs = np.ascontiguousarray(queries, dtype=np.int32)
    out = np.empty(max(qs.size, 1), dtype=np.float64)
    rc = _load().oracle_density_at(_ptr(X), X.shape[0], X.shape[1], X.shape[1], _ptr(qs), qs.size, float(r),
                                   _ptr(out))
    if rc < 0:
        raise ValueError("query row out of range")
    return out[:qs.size]


def lens_ecc_inf(X) -> np.ndarray:
    """Largest distance from each row to the cloud, O(n^2 d): small clouds
    only."""
    X = _f32(X)
    f = np.empty(X.shape[0], dtype=np.float64)
    _load().oracle_lens_ecc_inf(_ptr(X), X.shape[0], X.shape[1], X.shape[1], _ptr(f))
    return f


def lens_coord(X, j: int) -> np.ndarray:
    X = _f32(X)
    f = np.empty(X.shape[0], dtype=np.float64)
    _load().oracle_lens_coord(_ptr(X), X.shape[0], X.shape[1], X.shape[1], int(j), _ptr(f))
    return f


def lens_project(X, mu, v) -> np.ndarray:
    X = _f32(X)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    f = np.empty(X.shape[0], dtype=np.float64)
    _load().oracle_lens_project(_ptr(X), X.shape[0], X.shape[1], X.shape[1], _ptr(mu), _ptr(v), _ptr(f))
    return f


def pca(X, k: int = 1):
    """(mu, V[k, d], eigenvalues[k]) of the FP64 covariance (divide by n)."""
    X = _f32(X)
    d = X.shape[1]
    mu = np.empty(d, dtype=np.float64)
    V = np.empty((k, d), dtype=np.float64)
    lam = np.empty(k, dtype=np.float64)
    rc = _load().oracle_pca(_ptr(X), X.shape[0], d, d, int(k), _ptr(mu), _ptr(V), _ptr(lam))
    if rc < 0:
        raise RuntimeError(f"oracle_pca failed ({rc})")
    return mu, V, lam


def lens(X, kinds, args, pca_basis=None, radii=None) -> np.ndarray:
    """n x m lens. For principal-component lenses, `pca_basis` = (mu, V)
    fixes the projection (the GPU's own, for parity); otherwise the oracle's
    FP64 PCA supplies it. `radii[j]` is the ball radius of a density lens."""
    X = _f32(X)
    cols = []
    basis = pca_basis
    for kind, arg in zip(kinds, args):
        if kind == 0:
            cols.append(lens_l2(X))
        elif kind == 1:
            cols.append(lens_coord(X, arg))
        elif kind == 2:
            if basis is None:
                mu, V, _ = pca(X, max(a for kk, a in zip(kinds, args) if kk == 2) + 1)
                basis = (mu, V)
            cols.append(lens_project(X, basis[0], basis[1][arg]))
        elif kind == 3:
            cols.append(lens_ecc2(X))
        elif kind == 4:
            cols.append(lens_linf(X))
        elif kind == 5:
            cols.append(lens_density(X, radii[len(cols)]))
        elif kind == 6:
            cols.append(lens_ecc_inf(X))
        else:
            raise ValueError(kind)
    return np.ascontiguousarray(np.stack(cols, axis=1))


# ----------------------------------------------------------------- cover --

def interval_bounds(lo: float, hi: float, n_int: int, p: float):
    a = np.empty(n_int, dtype=np.float64)
    b = np.empty(n_int, dtype=np.float64)
    _load().oracle_interval_bounds(float(lo), float(hi), int(n_int), float(p), _ptr(a), _ptr(b))
    return a, b


def balanced_bounds(lens_col, n_int: int, p: float):
    """Interval bounds of the balanced cover of one filter column."""
    L = np.ascontiguousarray(lens_col, dtype=np.float64).reshape(-1)
    a = np.empty(n_int, dtype=np.float64)
    b = np.empty(n_int, dtype=np.float64)
    _load().oracle_balanced_bounds(_ptr(L), L.size, 1, 0, int(n_int), float(p), _ptr(a), _ptr(b))
    return a, b


def cover(lens_arr, n_intervals, overlap, balanced: bool = False):
    """(elem_offsets[E+1] int64, elem_points[sum n_i] int32); `balanced`:
    the balanced cover (uniform cover of the filter's ranks)."""
    L = np.ascontiguousarray(lens_arr, dtype=np.float64)
    if L.ndim == 1:
        L = L[:, None]
    n, m = L.shape
    ni = np.ascontiguousarray(n_intervals, dtype=np.int32)
    ov = np.ascontiguousarray(overlap, dtype=np.float64)
    E = int(np.prod(ni))
    offs = np.empty(E + 1, dtype=np.int64)
    lib = _load()
    total = lib.oracle_cover(_ptr(L), n, m, _ptr(ni), _ptr(ov), int(bool(balanced)), _ptr(offs), None)
    if total < 0:
        raise ValueError("bad cover arguments")
    pts = np.empty(max(total, 1), dtype=np.int32)
    lib.oracle_cover(_ptr(L), n, m, _ptr(ni), _ptr(ov), int(bool(balanced)), _ptr(offs), _ptr(pts))
    return offs, pts[:total]


# ---------------------------------------------------------------- DBSCAN --

def dbscan(X, pts, eps: float, min_pts: int):
    """DBSCAN on the rows `pts` (ascending) of X. Returns
    (count int32, core bool, label int64 [canonical id or -1], near_ties)."""
    X = _f32(X)
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    npt = pts.shape[0]
    count = np.zeros(max(npt, 1), dtype=np.int32)
    core = np.zeros(max(npt, 1), dtype=np.uint8)
    label = np.zeros(max(npt, 1), dtype=np.int64)
    ties = np.zeros(1, dtype=np.int64)
    _load().oracle_dbscan(_ptr(X), X.shape[0], X.shape[1], X.shape[1], _ptr(pts), npt,
                          float(eps), int(min_pts), _ptr(count), _ptr(core), _ptr(label), _ptr(ties))
    return count[:npt], core[:npt].astype(bool), label[:npt], int(ties[0])


# ----------------------------------------------------------- nodes, nerve --

def nodes_from_labels(elem_offsets, elem_points, labels):
    """Nodes ordered by (element, canonical id); members ascending.
    `labels` is aligned with elem_points (canonical id or -1).
    Returns node_offsets int64[N+1], node_members int32, node_elem int32."""
    E = len(elem_offsets) - 1
    offs = [0]
    members = []
    elems = []
    for e in range(E):
        s, t = int(elem_offsets[e]), int(elem_offsets[e + 1])
        lab = np.asarray(labels[s:t])
        pts = np.asarray(elem_points[s:t])
        for c in np.unique(lab[lab >= 0]):
            mem = np.sort(pts[lab == c])
            members.append(mem)
            elems.append(e)
            offs.append(offs[-1] + len(mem))
    node_members = (np.concatenate(members).astype(np.int32) if members
                    else np.zeros(0, dtype=np.int32))
    return (np.asarray(offs, dtype=np.int64), node_members, np.asarray(elems, dtype=np.int32))


def nerve(node_offsets, node_members, n_points: int):
    """1-skeleton of the nerve: edge {u, v}, u < v, iff some point lies in
    both nodes. Returns int32[E_g, 2], lexicographically sorted."""
    N = len(node_offsets) - 1
    if N == 0:
        return np.zeros((0, 2), dtype=np.int32)
    node_of = np.repeat(np.arange(N, dtype=np.int64), np.diff(node_offsets))
    pt = np.asarray(node_members, dtype=np.int64)
    order = np.lexsort((node_of, pt))          # group memberships by point
    pt, node_of = pt[order], node_of[order]
    us, vs = [], []
    start = 0
    while start < len(pt):
        end = start
        while end < len(pt) and pt[end] == pt[start]:
            end += 1
        ids = node_of[start:end]
        for a in range(len(ids)):
            for b in range(a + 1, len(ids)):
                us.append(ids[a]); vs.append(ids[b])
        start = end
    if not us:
        return np.zeros((0, 2), dtype=np.int32)
    key = np.unique(np.asarray(us, dtype=np.int64) * (N + 1) + np.asarray(vs, dtype=np.int64))
    return np.stack([key // (N + 1), key % (N + 1)], axis=1).astype(np.int32)


def mapper_graph(X, lens_arr, n_intervals, overlap, eps: float, min_pts: int,
                 elements=None, balanced: bool = False):
    """Full mapper graph from a given lens (n x m). With `elements` (a list
    of element indices) only those elements are clustered and the nerve is
    left empty (sampled parity at large sizes).

    Returns a dict: elem_offsets, elem_points, labels (per membership),
    core (per membership), counts, node_offsets, node_members, node_elem,
    edges, near_ties."""
    X = _f32(X)
    offs, pts = cover(lens_arr, n_intervals, overlap, balanced)
    E = len(offs) - 1
    labels = np.full(len(pts), -1, dtype=np.int64)
    core = np.zeros(len(pts), dtype=bool)
    counts = np.zeros(len(pts), dtype=np.int32)
    ties = 0
    todo = range(E) if elements is None else elements
    for e in todo:
        s, t = int(offs[e]), int(offs[e + 1])
        if t == s:
            continue
        c, k, lab, nt = dbscan(X, pts[s:t], eps, min_pts)
        counts[s:t], core[s:t], labels[s:t] = c, k, lab
        ties += nt
    out = dict(elem_offsets=offs, elem_points=pts, labels=labels, core=core,
               counts=counts, near_ties=ties)
    if elements is None:
        no, nm, ne = nodes_from_labels(offs, pts, labels)
        out.update(node_offsets=no, node_members=nm, node_elem=ne,
                   edges=nerve(no, nm, X.shape[0]))
    return out


# ------------------------------------------------------------- k-distance --

def knn_distance(X, queries, k: int) -> np.ndarray:
    """For each query row, the distance to its k-th nearest point of X (the
    point itself counted first, at distance 0)."""
    X = _f32(X)
    qs = np.ascontiguousarray(queries, dtype=np.int32)
    out = np.empty(max(qs.size, 1), dtype=np.float64)
    rc = _load().oracle_knn_distance(_ptr(X), X.shape[0], X.shape[1], X.shape[1], _ptr(qs), qs.size, int(k),
                                     _ptr(out))
    if rc < 0:
        raise ValueError("bad k-distance arguments")
    return out[:qs.size]


# ----------------------------------------------------------- single linkage --

def msf(X, pts, eps: float):
    """Minimum spanning forest of the eps-graph of the rows `pts`
    (ascending) of X: edges (u, v, d2) with u < v global indices, in the
    order of the key (d2, u, v) (Kruskal). The single-linkage dendrogram of
    the element, cut at eps."""
    X = _f32(X)
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    npt = pts.shape[0]
    u = np.empty(max(npt, 1), dtype=np.int32)
    v = np.empty(max(npt, 1), dtype=np.int32)
    d2 = np.empty(max(npt, 1), dtype=np.float64)
    k = _load().oracle_msf(_ptr(X), X.shape[0], X.shape[1], X.shape[1], _ptr(pts), npt, float(eps), _ptr(u),
                           _ptr(v), _ptr(d2))
    if k < 0:
        raise MemoryError("oracle_msf: out of memory")
    return u[:k], v[:k], d2[:k]


def single_linkage(pts, u, v, d2, h: float):
    """Single-linkage clusters at height h of one element: the components of
    the forest edges with d2 <= h * h; label per member = the smallest point
    index of its component (every point belongs to a cluster)."""
    pts = np.asarray(pts)
    pos = {int(p): i for i, p in enumerate(pts)}
    parent = list(range(len(pts)))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for a, b, w in zip(u, v, d2):
        if w <= h * h:
            ra, rb = find(pos[int(a)]), find(pos[int(b)])
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
    return np.array([int(pts[find(i)]) for i in range(len(pts))], dtype=np.int64)
