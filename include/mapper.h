/*
 * mapper.h -- C ABI of the GB300 mapper-graph library (libmapper_gb300.so).
 *
 * The library computes the mapper graph of "Mapper Interactive"
 * (arXiv 2011.03209), §3 Background: a filter (lens) f on a point cloud
 * X in R^d, a cover of f(X) by n overlapping intervals (or, for a 2D filter,
 * rectangles), DBSCAN(eps, minPts) on the points of each cover element, and
 * the 1D nerve of the resulting clusters (nodes = clusters, an edge between
 * two clusters that share a point). Every step runs in CUDA kernels written
 * for sm_103a (GB300); there is no CPU fallback.
 *
 * Conventions
 *   - Status: every int-returning call returns MAPPER_OK (0) or a negative
 *     mapper_status. Nothing aborts, exits or throws across this ABI. The
 *     message of the calling thread's last failure is mapper_last_error().
 *   - Pointers named *_dev are device pointers (cudaMalloc'd or torch CUDA
 *     storage on the context's device). Inputs are borrowed: the caller keeps
 *     them alive and unmodified until the call returns.
 *   - X is row-major FP32, n rows of d values, row stride ld >= d elements.
 *     X must be finite (MAPPER_ENONFINITE otherwise).
 *   - Results are library-owned opaque handles released with mapper_free().
 *     Their arrays are read with *_sizes() then *_copy() into caller-owned
 *     buffers, on the host (on_device = 0) or device (on_device = 1).
 *   - Calls are ordered on the context's stream. They return after the
 *     result is complete (sizes that shape an output are read back), so a
 *     handle is ready for *_copy when its call returns.
 *   - Threads: one context must not be used by two threads at once; distinct
 *     contexts are independent.
 *   - Result semantics (exact): graph, node memberships and edges equal those
 *     of the plain FP64 definition below, whatever the screening precision.
 *
 * Definitions (the readings where the paper is silent are fixed here):
 *   lens      L2: f(x) = sqrt(sum_k x_k^2), the exact sum rounded once to
 *             double, then a correctly rounded square root; COORD: f(x) = x_j;
 *             PCA: f(x) = sum_k (x_k - mu_k) v_k with v the j-th principal
 *             axis (double, k ascending, one rounding per operation); ECC:
 *             sqrt(mean_y |x - y|^2); LINF: max_k |x_k|; DENSITY: the number
 *             of points y with |x - y|^2 <= r*r (DBSCAN's distance); ECC_INF:
 *             max_y |x - y| (the DBSCAN distance, exact).
 *   cover     n intervals over [lo, hi] = [min f, max f]:
 *             L = (hi-lo)/(n-(n-1)p), s = L(1-p), a_k = lo + k s,
 *             b_k = a_k + L, then a_0 = lo, b_{n-1} = hi and
 *             b_k = max(b_k, a_{k+1}); L = 1 if hi == lo. Closed intervals.
 *             2D: element (i, j) has index i * n_2 + j.
 *   DBSCAN    q in N(p) iff sum_k (x_pk - x_qk)^2 <= eps*eps (double, k
 *             ascending) within one element; p in N(p); core iff
 *             |N(p)| >= minPts; clusters = components of the core points;
 *             canonical id = smallest point index among a cluster's cores; a
 *             non-core point with core neighbours joins the neighbouring
 *             cluster of smallest canonical id; others are noise.
 *   nodes     every cluster of every element, ordered by (element, canonical
 *             id); members in ascending point index.
 *   edges     {u, v}, u < v, iff nodes u and v share a point; sorted
 *             lexicographically.
 */
#ifndef MAPPER_GB300_H
#define MAPPER_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MAPPER_ABI_VERSION 6

typedef enum mapper_status {
    MAPPER_OK = 0,
    MAPPER_EINVAL = -1,      /* bad argument (sizes, parameters, null handle) */
    MAPPER_ENOMEM = -2,      /* device allocation failed or over the HBM budget */
    MAPPER_ECUDA = -3,       /* a CUDA runtime/driver call failed */
    MAPPER_ETIMEOUT = -4,    /* a bounded device-side wait ran out */
    MAPPER_ENONFINITE = -5,  /* X holds NaN or Inf */
    MAPPER_EINTERNAL = -6,   /* a device-side consistency check failed */
    MAPPER_ENOTIMPL = -7,    /* option not built in this library */
    MAPPER_ECANCELED = -8    /* a queued server request dropped by mapper_server_destroy */
} mapper_status;

typedef enum mapper_lens_kind {
    MAPPER_LENS_L2 = 0,      /* §3: "Common choices include the L2-norm" */
    MAPPER_LENS_COORD = 1,   /* §4.1: filter "based on a chosen dimension" */
    MAPPER_LENS_PCA = 2,     /* projection on a principal axis (PCA module, §4.1) */
    MAPPER_LENS_ECC = 3,     /* eccentricity, exponent 2: sqrt(mean over the cloud of
                                |x - y|^2) (§3 "eccentricity", §4.1 derived filters) */
    MAPPER_LENS_LINF = 4,    /* L-infinity norm max_k |x_k| (§5: the breast-cancer mapper
                                graphs filter by the "L_infinity-norm") */
    MAPPER_LENS_DENSITY = 5, /* density (§4.1 derived filters): the number of points within
                                distance r of x, x included, r = lens_param[j]; exact counts
                                (the pass-1 neighbour counts of DBSCAN(r, .) on the whole
                                cloud), returned as doubles */
    MAPPER_LENS_ECC_INF = 6  /* L-infinity centrality max_y |x - y| (§5 filters by the
                                "L_infinity-norm" of the pairwise distance matrix;
                                eccentricity with exponent infinity): the FP64 distance of the
                                defining expression, exact; O(n^2 d) */
} mapper_lens_kind;

/* Precision of the eps-neighbourhood screen. Every pair whose screened
 * distance falls inside a rigorous error band around eps^2 is re-decided in
 * FP64, so all precisions give the same exact graph. */
typedef enum mapper_precision {
    MAPPER_FP32 = 0,         /* CUDA-core FP32 sum of squared differences */
    MAPPER_BF16 = 1,         /* tcgen05 tensor cores, BF16 in, FP32 accumulate; rows
                                centred per group and split hi + lo: three products,
                                a narrow band */
    MAPPER_BF16X1 = 2,       /* as MAPPER_BF16 with the hi part only: one product, a
                                band about 2^8 times wider */
    MAPPER_FP8 = 3           /* count pass first on FP8 E4M3 tensor cores (kind::f8f6f4):
                                rows centred per group, scaled by one power of two per
                                128-row tile, split hi + lo (three products, FP32
                                accumulate); the 32 x 32 blocks with a pair in that band
                                are counted again with the three BF16 products of
                                MAPPER_BF16; the union pass is MAPPER_BF16's */
} mapper_precision;

typedef struct mapper_ctx mapper_ctx;
typedef struct mapper_cover_t mapper_cover_t;
typedef struct mapper_clusters_t mapper_clusters_t;
typedef struct mapper_graph_t mapper_graph_t;
typedef struct mapper_forest_t mapper_forest_t;

/* Parameters of one mapper graph (§3, "Algorithmic details in practice":
 * filter f, number of cover elements n, overlap p, metric, clusterer). */
/* Cover of the filter range (§3: "Each interval (cover element) typically has
 * uniform size"; some libraries offer a "balanced" cover whose intervals hold
 * equal numbers of points). */
typedef enum mapper_cover_kind {
    MAPPER_COVER_UNIFORM = 0,   /* n intervals of equal length over [min f, max f] */
    MAPPER_COVER_BALANCED = 1   /* the uniform cover of the ranks of f: with v_0 <= ..
                                   <= v_{n-1} the sorted values and [r_a, r_b] the uniform
                                   intervals over [0, n-1], the element is
                                   [v_ceil(r_a), v_min(floor(r_b), n-1)] (empty when
                                   ceil(r_a) > n-1), membership closed */
} mapper_cover_kind;

typedef struct mapper_params {
    int32_t m;               /* filter dimension: 1 (intervals) or 2 (rectangles) */
    int32_t lens_kind[2];    /* mapper_lens_kind per filter dimension */
    int32_t lens_arg[2];     /* COORD: column j; PCA: axis (0 = first); L2: ignored */
    int32_t n_intervals[2];  /* n >= 1 per filter dimension */
    double overlap[2];       /* p in [0, 1) per filter dimension */
    double eps;              /* DBSCAN radius, finite, > 0 */
    int32_t min_pts;         /* DBSCAN minPts >= 1 */
    int32_t precision;       /* mapper_precision */
    int32_t cover_kind;      /* mapper_cover_kind */
    double lens_param[2];    /* DENSITY: ball radius r (finite, > 0); other kinds: ignored */
} mapper_params;

/* Counters of one computation (filled by mapper_stats_get). */
typedef struct mapper_stats {
    int64_t n_points;        /* n */
    int64_t n_elements;      /* cover elements */
    int64_t n_members;       /* sum over elements of n_i */
    double sum_ni2;          /* sum over elements of n_i^2 */
    int64_t tile_pairs;      /* candidate tile pairs (both tiles in one element) */
    int64_t tile_pairs_out;  /* ... certified all-out by bounding spheres (skipped) */
    int64_t tile_pairs_in;   /* ... certified all-in by bounding spheres (no distances) */
    int64_t pairs_screened;  /* point pairs evaluated by the screen, all passes */
    int64_t band_pairs;      /* pairs in the band of the first screen, all passes */
    int64_t near_ties;       /* unordered pairs with |d^2 - eps^2| <= 1e-12 eps^2 */
    int64_t n_core;          /* core memberships */
    int64_t n_nodes;
    int64_t n_edges;
    int64_t n_launches;      /* kernels this call launched */
    double ms_lens, ms_cover, ms_cluster, ms_nerve, ms_total;  /* device time (timing on) */
    double ms_pass[3];       /* device time of the count, union and border passes */
    double ms_tiles;         /* device time of tile layout and tile-pair classification */
    int64_t tile_pairs_tc;   /* mixed tile pairs screened on tensor cores */
    int64_t tile_pairs_simt; /* mixed tile pairs across two segments (two centres): CUDA cores
                                (FP32), or tensor cores (tile_pairs_cross) */
    int64_t union_skipped;   /* union-pass tile pairs skipped: their cores already joined */
    int64_t n_groups;        /* pivot groups of the tile layout */
    int64_t n_rows;          /* rows of the tile layout (memberships + tile padding) */
    int64_t count_kernel_pairs;  /* point pairs screened by the main count kernel: the
                                    tensor-core one (BF16 precisions) or the CUDA-core
                                    one (FP32) */
    double ms_count_kernel;  /* device time of that kernel's launch (timing on) */
    int64_t union_pairs;     /* screened tile pairs with a neighbour pair, given to the union
                                pass (before its rounds skip joined ones) */
    int64_t fp64_pairs;      /* pairs decided by the FP64 defining expression, all passes */
    int64_t pass1_tile_n;    /* N of the pass-1 tensor-core product, picked by the context's
                                autotuner: 128 (one tile pair per work item) or 256 (two tile
                                pairs sharing tile A); 0 off the tensor cores */
    int64_t tile_pairs_cross;  /* of tile_pairs_simt (mixed pairs across two segments of one
                                  element), those screened on the tensor cores with rows
                                  centred per element: all of them when they are at least
                                  1/32 of the rows (BF16 precisions), else none */
    int64_t tile_pairs_screen1;  /* MAPPER_BF16 two-phase count pass: tile pairs screened first
                                    with one product (hi.hi); 0 when every pair took three */
    int64_t tile_pairs_redo;     /* ... of them, the tile pairs with a pair inside the
                                    one-product band, screened again with three products */
    int64_t redo_blocks;         /* ... the 32 x 32 blocks of those pairs that hold one */
    int64_t redo_parts;          /* ... the 32-column parts of those pairs holding such a block */
    int64_t pass1_phases;        /* phases of the tensor-core count pass: 2 (a first screen, then
                                    three products for its deferred blocks) or 1 (three products);
                                    0 off the tensor cores */
    double pass1_sample_deferred; /* pass-1 screen 0: the fraction of a sample of the tile pairs
                                     whose first screen deferred a block; -1 when no sample ran.
                                     MAPPER_BF16: one phase or two, and the pairs sent straight to
                                     three products, follow the sample's fractions per bin of the
                                     tile-pair statistic below; MAPPER_FP8: one phase above 0.35 */
    int64_t tile_pairs_direct;    /* pass-1 screen 0, two phases (MAPPER_BF16): tensor-core tile
                                     pairs sent straight to three products, those whose bin of
                                     (|c_a - c_b|^2 + r_a^2 + r_b^2) / eps^2 (tile spheres) deferred
                                     a block in at least half of its sampled pairs */
} mapper_stats;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`, ordering all work on
 * `cuda_stream` (a cudaStream_t; NULL = a stream the context creates).
 * hbm_budget_bytes caps the context's scratch (0 = no cap). When the
 * environment variable MAPPER_TUNE_CACHE names a file, the context starts
 * from the pass-1 shapes the autotuner chose before on the same kind of
 * device (device name and SM count) and mapper_destroy merges its own
 * choices into the file. */
int mapper_create(mapper_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream);
void mapper_destroy(mapper_ctx* ctx);
/* Use another stream for subsequent calls. */
int mapper_set_stream(mapper_ctx* ctx, void* cuda_stream);
/* Record per-stage device times in mapper_stats (adds CUDA events). */
int mapper_set_timing(mapper_ctx* ctx, int enabled);
/* Shape of the pass-1 tensor-core product (a tuning knob; the paper has no
 * counterpart and results do not depend on it): 0 = let the context's
 * autotuner pick per row pitch and screen (default), 128 = one tile pair per
 * work item, 256 = two tile pairs sharing their first tile. Other values:
 * MAPPER_EINVAL. */
int mapper_set_pass1_tile_n(mapper_ctx* ctx, int tile_n);
/* Count-pass screen of MAPPER_BF16 and MAPPER_FP8 (a tuning knob; results do
 * not depend on it): 0 = the default: per call, the first screen of mode 3
 * on every 64th tile pair decides (two phases of mode 3 unless more than 35 %
 * of those pairs defer a block, then one phase), 1 = two phases: every tile pair
 * first with one BF16 product (hi.hi, the band of MAPPER_BF16X1), or three
 * FP8 products; each 32 x 32 block of a tile pair that has a pair inside
 * that band is counted by a second pass with three BF16 products, the others
 * are final after the first, 2 = one phase: three products (BF16, or FP8
 * with its band re-decided in FP64) for every tile pair, 3 = two phases where
 * the first defers every block with a row that its extremes do not decide
 * (all in or all out) without screening its values. Other values:
 * MAPPER_EINVAL. */
int mapper_set_pass1_screen(mapper_ctx* ctx, int mode);
/* Where the BF16 precisions screen mixed tile pairs across two segments of
 * one element (a tuning knob; results do not depend on it): 0 = on the
 * tensor cores when they are at least 1/32 of the rows, else on CUDA cores
 * (default), 1 = always on the tensor cores (rows centred per element, a
 * second operand set), 2 = always on CUDA cores. Other values: MAPPER_EINVAL. */
int mapper_set_cross_screen(mapper_ctx* ctx, int mode);
/* Capacity of the tensor-core screen's band queue, in pairs (a tuning and
 * testing knob; the paper has no counterpart and results do not depend on
 * it): band pairs past the capacity are decided in FP64 inside the screen
 * kernel instead of by the separate recheck. 0 = sized from the tile pairs
 * (2^20 to 2^25 entries, the default); 1 .. 2^30 = that many entries.
 * Other values: MAPPER_EINVAL. */
int mapper_set_band_queue_cap(mapper_ctx* ctx, int64_t entries);
/* Failure-detection self-test (the paper has no counterpart): runs the
 * bounded mbarrier wait of the tensor-core passes on a barrier that nothing
 * completes. Returns MAPPER_ETIMEOUT after the wait's limit (4 s), the status
 * a pass reports when a wait runs out; the context stays usable. */
int mapper_selftest_wait(mapper_ctx* ctx);
/* Accumulation self-test of the tensor-core screen (the paper has no
 * counterpart): random rows of row pitch dp (a multiple of 32 in [32, 4096])
 * through the screen's tcgen05 products (1: hi.hi, 3: hi.hi + hi.lo + lo.hi)
 * for four 128 x 128 tile pairs; format 0 = BF16 parts (magnitudes 2^-4 ..
 * 2^5, kind::f16), 1 = FP8 E4M3 parts (hi 2^-4 .. 2^5, lo 2^-8 .. 2^1,
 * kind::f8f6f4). *observed = the largest |accumulator - exact sum| over them,
 * relative to the sum of the magnitudes of the products; *modelled = the
 * accumulation term the screen's error bound assumes, relative to the same
 * sum (BF16: (dp / 16 * products + 8) units of 2^-22, times (1 + 2u')^2;
 * FP8: (dp / 32 * products + 8) units, times 1.3). The bound is sound on
 * this hardware only if observed stays below modelled. */
int mapper_selftest_mma_error(mapper_ctx* ctx, int32_t dp, int32_t products, int32_t format, uint64_t seed,
                              double* observed, double* modelled);
/* Screen of mapper_knn_distance (a tuning knob; results do not depend on
 * it): 0 = tensor cores (default), 1 = tensor cores, 2 = the FP32 CUDA-core
 * screen, 3 = tensor cores without the sampled threshold (per-part lists
 * only). Other values: MAPPER_EINVAL. */
int mapper_set_knn_screen(mapper_ctx* ctx, int mode);
/* The path the context's last mapper_knn_distance call took, in info[8]:
 * [0] 0 = CUDA-core screen, 1 = tensor-core list screen, 2 = tensor-core
 * screen with a threshold per query from a sample of the points (clouds of
 * at least 512 tiles of 128 points; k <= 8); [1] the queries whose keys
 * below their threshold exceeded the capacity and went through the list
 * screen; [2] that capacity (keys per query); [3] the sample's tile stride;
 * [4] the keys below the thresholds (all queries); [5] the largest such count
 * of one query; [6] the candidates whose FP32 distance the merge computed;
 * [7] those given the FP64 defining expression. Tensor-core paths fill
 * [6] and [7]; the sampled path [1] .. [5]. Zeros before the first call.
 * MAPPER_EINVAL for null arguments. */
int mapper_knn_info(const mapper_ctx* ctx, int64_t* info);

/* -------------------------------------------------------------- the steps */

/* Lens (§3 filter function; §4.1 L2 norm / chosen column; PCA module).
 * Writes lens_dev[p * m + j] = f_j(x_p) for p < n, j < m (caller-owned,
 * device, n*m doubles). kinds[j], args[j] as in mapper_params (host arrays).
 * For PCA lenses, pca_out (optional, host) receives mu[d] followed by the
 * axes v_0..v_{K-1} (K = 1 + largest PCA axis asked for), each d doubles;
 * the axes come from power iteration on the FP32 covariance, each signed
 * so its entry of largest magnitude is positive. */
int mapper_lens(mapper_ctx* ctx, const float* X_dev, int64_t n, int32_t d, int64_t ld,
                int32_t m, const int32_t* kinds, const int32_t* args,
                double* lens_dev, double* pca_out);
/* The same with per-dimension real parameters lens_param[m] (host; the
 * density radius; may be NULL when no lens needs one) and the screen
 * precision of the density lens's neighbour counts (mapper_precision; the
 * counts are exact in every precision). mapper_lens is this call with
 * lens_param = NULL and MAPPER_BF16. A density lens without a finite radius
 * > 0: MAPPER_EINVAL. */
int mapper_lens_ex(mapper_ctx* ctx, const float* X_dev, int64_t n, int32_t d, int64_t ld,
                   int32_t m, const int32_t* kinds, const int32_t* args, const double* lens_param,
                   int32_t precision, double* lens_dev, double* pca_out);

/* Cover (§3: intervals V_k of f(X), n elements, overlap p; 2D: rectangles)
 * and pull-back: for each element, the points with f in it, ascending.
 * lens_dev: n*m doubles (device, row-major). n_intervals, overlap: host
 * arrays of m. Result read with mapper_cover_sizes / mapper_cover_copy. */
int mapper_cover(mapper_ctx* ctx, const double* lens_dev, int64_t n, int32_t m,
                 const int32_t* n_intervals, const double* overlap, mapper_cover_t** out);
/* The same with the balanced cover (mapper_cover_kind). */
int mapper_cover_balanced(mapper_ctx* ctx, const double* lens_dev, int64_t n, int32_t m,
                          const int32_t* n_intervals, const double* overlap, mapper_cover_t** out);
int mapper_cover_sizes(const mapper_cover_t* cover, int64_t* n_elements, int64_t* n_members);
/* elem_offsets: n_elements+1 int64; elem_points: n_members int32. */
int mapper_cover_copy(const mapper_cover_t* cover, int64_t* elem_offsets, int32_t* elem_points,
                      int on_device);

/* DBSCAN(eps, minPts) inside every element of `cover` (§3; the per-element
 * decomposition is the parallelisation of §4.3). X must be the cloud the
 * cover's lens was computed on. Result read with mapper_clusters_copy. */
int mapper_cluster(mapper_ctx* ctx, const float* X_dev, int64_t n, int32_t d, int64_t ld,
                   const mapper_cover_t* cover, double eps, int32_t min_pts, int32_t precision,
                   mapper_clusters_t** out);
/* Per membership slot (aligned with the cover's elem_points): label =
 * canonical cluster id or -1 (noise); core = 1 if core. Either may be NULL. */
int mapper_clusters_copy(const mapper_clusters_t* clusters, int64_t* label, uint8_t* core,
                         int on_device);

/* Single linkage (§5: Lum et al. cluster each cover element by single
 * linkage, where the tool uses DBSCAN). For every element of `cover`, the
 * minimum spanning forest of its eps-graph: the points of the element, an
 * edge {p, q} where d2(p, q) <= eps*eps (the DBSCAN distance of this
 * header), edges ordered by the key (d2, smaller point index, larger point
 * index), so the forest is unique when distances tie. Equivalently, the
 * single-linkage dendrogram of the element up to height eps. The result is
 * read with mapper_forest_sizes / mapper_forest_copy: edge k joins points
 * u[k] < v[k] of element elem[k] at squared distance d2[k] (the FP64 value of
 * the defining expression); edges come in no particular order (sort by
 * (elem, d2, u, v) for a canonical one). X must be the cloud the cover was
 * built on. MAPPER_EINVAL for eps not finite and > 0, MAPPER_ENONFINITE if X
 * holds NaN/Inf. */
int mapper_single_linkage(mapper_ctx* ctx, const float* X_dev, int64_t n, int32_t d, int64_t ld,
                          const mapper_cover_t* cover, double eps, mapper_forest_t** out);
int mapper_forest_sizes(const mapper_forest_t* forest, int64_t* n_edges);
/* elem, u, v: n_edges int32 each; d2: n_edges doubles. Any may be NULL. */
int mapper_forest_copy(const mapper_forest_t* forest, int32_t* elem, int32_t* u, int32_t* v, double* d2,
                       int on_device);
/* Single-linkage clusters at height h, 0 < h <= the forest's eps: in every
 * element, the components of its forest edges with d2 <= h*h; every point is
 * a member of its component's cluster (no noise), whose canonical id is the
 * component's smallest point index. The handle is read like mapper_cluster's
 * (every point flagged core) and mapper_nerve builds its mapper graph, which
 * equals the graph of DBSCAN(h, minPts = 1). */
int mapper_forest_cut(mapper_ctx* ctx, const mapper_forest_t* forest, double h, mapper_clusters_t** out);

/* Nerve (§3: 1D nerve; an edge where two clusters intersect). */
int mapper_nerve(mapper_ctx* ctx, const mapper_clusters_t* clusters, mapper_graph_t** out);

/* Element sharding across GPUs (§4.3: the clustering of each cover element
 * is independent; §6 names distributing it across several GPUs, with the
 * merge of results, as the next step). A rank clusters a subset of the
 * elements, the ranks exchange their nodes, and every rank builds the nerve
 * of the merged node list.
 *
 * mapper_cover_subset: a cover holding only elements[0 .. k) of `cover`
 * (host int32 indices, distinct, in [0, n_elements)), renumbered 0 .. k-1 in
 * the given order, each with its points ascending as before. The result is
 * a new cover handle (release with mapper_free); MAPPER_EINVAL for an index
 * out of range or repeated.
 *
 * mapper_nerve_from_nodes: a graph whose nodes are given (node u = members
 * node_members[node_offsets[u] .. node_offsets[u+1]) of points in
 * [0, n_points), ascending, and node_elem[u] its element) and whose edges
 * are computed here as in mapper_nerve. The three arrays may be host or
 * device pointers (all of one kind) and are copied; node_offsets has
 * n_nodes + 1 entries starting at 0. The graph has no lens, cover or
 * clusters (mapper_graph_cover / _clusters return NULL). */
int mapper_cover_subset(mapper_ctx* ctx, const mapper_cover_t* cover, const int32_t* elements, int32_t k,
                        mapper_cover_t** out);
int mapper_nerve_from_nodes(mapper_ctx* ctx, int64_t n_points, int64_t n_nodes, const int64_t* node_offsets,
                            const int32_t* node_members, const int32_t* node_elem, mapper_graph_t** out);

/* k-th nearest-neighbour distances (§5: a module plots the distribution of
 * the distances to the k-th nearest neighbours, k = 5, to choose eps): for
 * each query row index queries[i] (in [0, n)), the k-th smallest distance to
 * the rows of X, the row itself counted first (distance 0), so the row is
 * core for DBSCAN(eps, k) on the whole cloud iff the value is <= eps. The
 * value is the FP64 distance of the defining expression (double sum of
 * squared differences, k ascending, sqrt), found exactly through a screen
 * (tensor cores, BF16 hi + lo products of rows centred on the column means,
 * or FP32 CUDA cores; mapper_set_knn_screen) and an FP64 decision of its
 * candidates. X: device memory. queries (q int32) and out (q doubles): host or
 * device memory, out filled before the call returns. k in [1, min(16, n)];
 * MAPPER_EINVAL otherwise, MAPPER_ENONFINITE if X holds NaN/Inf. */
int mapper_knn_distance(mapper_ctx* ctx, const float* X_dev, int64_t n, int32_t d, int64_t ld,
                        const int32_t* queries, int64_t q, int32_t k, double* out);

/* Fused call: lens, cover, cluster and nerve in one. X may be a device
 * pointer or a host pointer (pinned or pageable); a host X is copied to the
 * device inside the call. */
int mapper_graph(mapper_ctx* ctx, const float* X, int64_t n, int32_t d, int64_t ld,
                 const mapper_params* params, mapper_graph_t** out);

/* Parameter sweep (§4.4: the command line computes graphs over ranges of
 * parameters): n_sweep graphs of one cloud, graph i with radius eps[i] and
 * overlap[i] (for every filter dimension), the other parameters from
 * `params`. The lens is computed once, the cover and the tile layout once per
 * distinct overlap and shared by its radii; on the BF16 screens (MAPPER_BF16,
 * MAPPER_BF16X1) up to four distinct radii of one overlap also share one
 * count pass (one contraction, each radius decided in its epilogue). out:
 * n_sweep handles (each released with mapper_free; graphs of equal (eps,
 * overlap) share their clusters). Results equal n_sweep mapper_graph calls. */
int mapper_graph_sweep(mapper_ctx* ctx, const float* X, int64_t n, int32_t d, int64_t ld,
                       const mapper_params* params, int32_t n_sweep, const double* eps, const double* overlap,
                       mapper_graph_t** out);

int mapper_graph_sizes(const mapper_graph_t* g, int64_t* n_nodes, int64_t* n_members,
                       int64_t* n_edges);
/* node_offsets: n_nodes+1 int64; node_members: n_members int32; node_elem:
 * n_nodes int32 (cover element of each node); edges: 2*n_edges int32
 * (u, v pairs). Any pointer may be NULL to skip that array. */
int mapper_graph_copy(const mapper_graph_t* g, int64_t* node_offsets, int32_t* node_members,
                      int32_t* node_elem, int32_t* edges, int on_device);
/* The lens the graph was built from (n*m doubles), its PCA basis if any
 * (mu then axes, d doubles each; returns the count of doubles written via
 * *n_pca, 0 if no PCA lens), and the cover it used. */
int mapper_graph_lens(const mapper_graph_t* g, double* lens, double* pca, int64_t* n_pca,
                      int on_device);
const mapper_cover_t* mapper_graph_cover(const mapper_graph_t* g);
const mapper_clusters_t* mapper_graph_clusters(const mapper_graph_t* g);

/* Counters of a clusters, graph or forest handle. */
int mapper_stats_get(const void* handle, mapper_stats* out);

/* Release any handle (cover, clusters, graph, forest). NULL is a no-op. */
void mapper_free(void* handle);

/* ------------------------------------------------------------- serving */

/* Estimated device bytes one mapper_graph call on an n x d cloud with these
 * parameters holds at its peak (for admission control; not a guarantee). */
int mapper_graph_footprint(int64_t n, int32_t d, const mapper_params* params, size_t* bytes);

/* A request server (§4.1: the interface recomputes the graph whenever a
 * parameter changes; §4.4: parameter ranges computed offline). Datasets stay
 * resident on the device; requests (dataset, parameters) are queued in
 * arrival order. A free one of n_slots worker slots starts the oldest queued
 * request whose estimated footprint fits in hbm_budget_bytes beside the
 * running ones (0 = 80 % of the device's free memory at creation); when
 * nothing runs, the oldest request starts whatever its size. A younger
 * request that fits may overtake an older one that does not, at most 8 times
 * per older request; then the slots wait for the older one. Each slot is a
 * host thread with its own context and CUDA stream, so running requests
 * overlap on the device. Results are the exact graphs of mapper_graph.
 * Thread-safe. */
typedef struct mapper_server mapper_server;

typedef struct mapper_request_info {
    double queue_s;          /* submit -> start of work */
    double run_s;            /* start of work -> graph ready */
    double latency_s;        /* submit -> graph ready */
    size_t footprint;        /* the admission estimate it ran under */
    int32_t status;          /* mapper_status of the computation */
} mapper_request_info;

int mapper_server_create(mapper_server** out, int device, int n_slots, size_t hbm_budget_bytes);
/* Stops the slots after their running requests. Requests still queued are
 * dropped: their waiters return MAPPER_ECANCELED. Returns after every thread
 * inside mapper_server_wait has returned; the server must not be used after
 * this call starts (a wait that begins afterwards is invalid). */
void mapper_server_destroy(mapper_server* server);
/* X_dev: device FP32 cloud (n rows, stride ld), borrowed until destroy. */
int mapper_server_add_dataset(mapper_server* server, const float* X_dev, int64_t n, int32_t d, int64_t ld,
                              int32_t* dataset_id);
int mapper_server_submit(mapper_server* server, int32_t dataset_id, const mapper_params* params,
                         int64_t* request_id);
/* Waits for a request (timeout_s < 0: no limit; MAPPER_ETIMEOUT otherwise)
 * and hands its graph to the caller (release with mapper_free). info may be
 * NULL. A request is collected once. */
int mapper_server_wait(mapper_server* server, int64_t request_id, double timeout_s, mapper_graph_t** out,
                       mapper_request_info* info);
int mapper_server_load(mapper_server* server, int* running, int* queued, size_t* bytes_in_use);

/* ----------------------------------------------- allocation-free variant */

/* DBSCAN(eps, minPts) of one point set, allocating no device memory.
 * The paper has no counterpart: this entry point serves callers that cannot
 * call cudaMalloc -- code hosted by a framework that owns every device
 * allocation through a fixed memory plan and forbids its plug-ins to
 * allocate, or latency-critical code that must never let an allocation
 * synchronise the device or fail half way through.
 *
 * Computes the same per-element DBSCAN as mapper_cluster (FP32 screen, FP64
 * re-decision of the error band, so results equal the FP64 definition
 * above) with the n rows of X_dev as the single element:
 *   label_dev[p] (device, n int64): canonical cluster id = smallest row index
 *                among the cluster's core points, or -1 for noise;
 *   core_dev[p]  (device, n uint8, may be NULL): 1 if row p is a core point.
 * X_dev, label_dev and core_dev are caller-owned device memory on the
 * calling thread's current device; work is ordered on cuda_stream (a
 * cudaStream_t, NULL = the legacy default stream) and the call returns after
 * it completes.
 *
 * Scratch lives in one fixed device array inside the library (about 8.6 MB,
 * held by every GPU that loads the library until the process exits), so
 * sizes are limited: n <= MAPPER_NOALLOC_MAX_POINTS and
 * d <= MAPPER_NOALLOC_MAX_DIM; larger inputs return MAPPER_EINVAL before any
 * GPU work. The first call in a CUDA context (normally the device's primary
 * context) looks up the array's device address there (cudaGetSymbolAddress)
 * and caches it under the context's unique id, so the address is valid for
 * that context's lifetime and a context created again gets a new lookup.
 * The call waits
 * for its stream (it reads a status word back before returning). Every call
 * shares the array and clears what must start at zero itself; calls that
 * overlap on the GPU (two streams, two threads) race on it and must be
 * ordered by the caller. A call that fails after queuing kernels waits for
 * them before it returns.
 * Errors: MAPPER_EINVAL (sizes, eps, minPts, a null X_dev or label_dev, or
 * X_dev, label_dev or a non-null core_dev that is not device memory of the
 * current device), MAPPER_ENONFINITE (X holds NaN/Inf), MAPPER_ECUDA. */
#define MAPPER_NOALLOC_MAX_POINTS 8192
#define MAPPER_NOALLOC_MAX_DIM 256
int mapper_dbscan_noalloc(const float* X_dev, int64_t n, int32_t d, int64_t ld, double eps,
                          int32_t min_pts, int64_t* label_dev, uint8_t* core_dev,
                          void* cuda_stream);

const char* mapper_strerror(int status);
const char* mapper_last_error(void);
int mapper_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MAPPER_GB300_H */
