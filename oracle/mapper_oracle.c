/*
 * mapper_oracle.c -- FP64 reference implementation of the mapper graph.
 *
 * TEST INFRASTRUCTURE ONLY. The test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library; the product (CUDA) path
 * never does, and it shares no code, header, table or constant with it.
 *
 * It follows "Mapper Interactive" (arXiv 2011.03209), §3 Background:
 *   1. a filter (lens) f on the point cloud X in R^d            (§3, §4.1)
 *   2. a cover of f(X) by n intervals with overlap fraction p    (§3)
 *      (for a 2D filter, rectangles: products of two covers)     (§3)
 *   3. DBSCAN(eps, minPts) on the points of each cover element   (§3)
 *   4. the 1D nerve: nodes = clusters, edge iff two share a point (§3)
 * Steps 1-3 live here; step 4 and node numbering are in oracle/__init__.py.
 * Beside the graph: further filters (eccentricity, L-infinity norm and
 * centrality, density; §3, §4.1, §5) and the k-th nearest-neighbour distance
 * of §5's module for choosing eps.
 *
 * Every step is written in its most direct form: brute-force O(n_i^2)
 * distances in double precision, breadth-first search for connected
 * components, no blocking, tiling or reordering. The file is compiled with
 * -ffp-contract=off so each written operation rounds once.
 *
 * Readings where the paper is silent (the same readings bind the CUDA path):
 *   - interval k of n over [lo, hi]: L = (hi-lo) / (n - (n-1) p),
 *     s = L (1-p), a_k = lo + k s, b_k = a_k + L; then a_0 = lo,
 *     b_{n-1} = hi, and b_k = max(b_k, a_{k+1}) so rounding opens no gap;
 *     if hi == lo then L = 1. Membership is closed: a_k <= f <= b_k.
 *   - 2D element (i, j) has index i * n_2 + j.
 *   - q is a neighbour of p iff sum_k (x_pk - x_qk)^2 <= eps * eps, summed
 *     in double for k ascending; p is its own neighbour; p is core iff it
 *     has at least minPts neighbours.
 *   - clusters are the connected components of the core points under the
 *     neighbour relation; a cluster's canonical id is the smallest global
 *     index among its core points; a non-core point with core neighbours
 *     joins the neighbouring cluster of smallest canonical id; the rest is
 *     noise in that element.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ---------------------------------------------------------------- lens -- */

/* L2-norm filter (§3 "Common choices include the L2-norm"; §4.1 control
 * panel): f(x) = sqrt(sum_k x_k^2), k ascending, in double. */
void oracle_lens_l2(const float* X, int64_t n, int32_t d, int64_t ld, double* f)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; ++p) {
        const float* x = X + p * ld;
        double s = 0.0;
        for (int32_t k = 0; k < d; ++k) {
            double v = (double)x[k];
            s = s + v * v;
        }
        f[p] = sqrt(s);
    }
}

/* Eccentricity filter (§3 lists eccentricity among the common filters;
 * §4.1 offers it beside the L2 norm and density), exponent 2:
 *   f(x) = ( (1/n) sum_{y in X} d(x, y)^2 )^(1/2),
 * d the Euclidean distance. Direct O(n^2 d) form: for each x, the squared
 * distances summed over y ascending (each a k-ascending double sum), divided
 * by n, square root. */
void oracle_lens_ecc2(const float* X, int64_t n, int32_t d, int64_t ld, double* f)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < n; ++p) {
        const float* x = X + p * ld;
        double s = 0.0;
        for (int64_t q = 0; q < n; ++q) {
            const float* y = X + q * ld;
            double d2 = 0.0;
            for (int32_t k = 0; k < d; ++k) {
                double t = (double)x[k] - (double)y[k];
                d2 = d2 + t * t;
            }
            s = s + d2;
        }
        f[p] = sqrt(s / (double)n);
    }
}

/* L-infinity-norm filter (§5, breast-cancer use case: the first filter of
 * both 2D mapper graphs is the "L_infinity-norm"). Reading: the norm of the
 * point itself, f(x) = max_k |x_k|, as L2 is sqrt(sum_k x_k^2). */
void oracle_lens_linf(const float* X, int64_t n, int32_t d, int64_t ld, double* f)
{
    for (int64_t p = 0; p < n; ++p) {
        const float* x = X + p * ld;
        double m = 0.0;
        for (int32_t k = 0; k < d; ++k) {
            double v = fabs((double)x[k]);
            if (v > m) m = v;
        }
        f[p] = m;
    }
}

/* Density filter (§4.1 lists density among the derived filters; no estimator
 * is given). Reading: the number of points of the cloud within distance r of
 * x, x itself included (a ball-count, i.e. uniform-kernel, density estimate
 * without its constant factor): f(x) = |{y in X : d(x, y)^2 <= r * r}|, the
 * squared distance summed in double for k ascending as in DBSCAN. */
void oracle_lens_density(const float* X, int64_t n, int32_t d, int64_t ld, double r, double* f)
{
    const double r2 = r * r;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < n; ++p) {
        const float* x = X + p * ld;
        int64_t c = 0;
        for (int64_t q = 0; q < n; ++q) {
            const float* y = X + q * ld;
            double d2 = 0.0;
            for (int32_t k = 0; k < d; ++k) {
                double t = (double)x[k] - (double)y[k];
                d2 = d2 + t * t;
            }
            if (d2 <= r2) ++c;
        }
        f[p] = (double)c;
    }
}

/* The density filter at the points queries[0..q) only (sampled parity at
 * sizes where all n^2 pairs are too many): out[i] = f(x_queries[i]) with f
 * as in oracle_lens_density. Returns -1 for a query outside [0, n). */
int oracle_density_at(const float* X, int64_t n, int32_t d, int64_t ld, const int32_t* queries, int64_t q,
                      double r, double* out)
{
    const double r2 = r * r;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < q; ++i) {
        if (queries[i] < 0 || queries[i] >= n) { bad = 1; continue; }
        const float* x = X + (int64_t)queries[i] * ld;
        int64_t c = 0;
        for (int64_t y = 0; y < n; ++y) {
            const float* yv = X + y * ld;
            double d2 = 0.0;
            for (int32_t k = 0; k < d; ++k) {
                double t = (double)x[k] - (double)yv[k];
                d2 = d2 + t * t;
            }
            if (d2 <= r2) ++c;
        }
        out[i] = (double)c;
    }
    return bad ? -1 : 0;
}

/* L-infinity centrality, the other reading of §5's "L_infinity-norm" filter
 * computed from the pairwise distance matrix: the largest entry of x's row,
 * f(x) = max_{y in X} d(x, y) (eccentricity with exponent infinity). The
 * largest squared distance (double sum, k ascending), then sqrt. */
void oracle_lens_ecc_inf(const float* X, int64_t n, int32_t d, int64_t ld, double* f)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < n; ++p) {
        const float* x = X + p * ld;
        double m = 0.0;
        for (int64_t q = 0; q < n; ++q) {
            const float* y = X + q * ld;
            double d2 = 0.0;
            for (int32_t k = 0; k < d; ++k) {
                double t = (double)x[k] - (double)y[k];
                d2 = d2 + t * t;
            }
            if (d2 > m) m = d2;
        }
        f[p] = sqrt(m);
    }
}

/* Filter "based on a chosen dimension (column)" (§4.1): f(x) = x_j. */
void oracle_lens_coord(const float* X, int64_t n, int32_t d, int64_t ld, int32_t j, double* f)
{
    (void)d;
    for (int64_t p = 0; p < n; ++p) f[p] = (double)X[p * ld + j];
}

/* Projection filter f(x) = sum_k (x_k - mu_k) v_k, k ascending, in double.
 * Used for the principal-component lens with a given (mu, v). */
void oracle_lens_project(const float* X, int64_t n, int32_t d, int64_t ld,
                         const double* mu, const double* v, double* f)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; ++p) {
        const float* x = X + p * ld;
        double s = 0.0;
        for (int32_t k = 0; k < d; ++k) {
            double t = (double)x[k] - mu[k];
            s = s + t * v[k];
        }
        f[p] = s;
    }
}

/* Principal components (PCA is one of the paper's analysis modules, §4.1;
 * it serves here as a lens). mean mu_j = (1/n) sum_p x_pj; covariance
 * C_jl = (1/n) sum_p (x_pj - mu_j)(x_pl - mu_l); eigenpairs of C by the
 * cyclic Jacobi method; the top-k eigenvectors in decreasing eigenvalue
 * order, each signed so that its entry of largest magnitude is positive
 * (ties: smallest index). V is k x d row-major. Returns the sweep count, or
 * -1 if Jacobi did not converge in 100 sweeps. */
int oracle_pca(const float* X, int64_t n, int32_t d, int64_t ld, int32_t k,
               double* mu, double* V, double* lambda)
{
    if (k < 1 || k > d || n < 1) return -3;
    double* C = (double*)calloc((size_t)d * d, sizeof(double));
    double* E = (double*)calloc((size_t)d * d, sizeof(double));
    if (!C || !E) { free(C); free(E); return -2; }

    for (int32_t j = 0; j < d; ++j) {
        double s = 0.0;
        for (int64_t p = 0; p < n; ++p) s = s + (double)X[p * ld + j];
        mu[j] = s / (double)n;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t j = 0; j < d; ++j) {
        for (int32_t l = j; l < d; ++l) {
            double s = 0.0;
            for (int64_t p = 0; p < n; ++p) {
                double a = (double)X[p * ld + j] - mu[j];
                double b = (double)X[p * ld + l] - mu[l];
                s = s + a * b;
            }
            C[(size_t)j * d + l] = s / (double)n;
            C[(size_t)l * d + j] = s / (double)n;
        }
    }
    for (int32_t j = 0; j < d; ++j) E[(size_t)j * d + j] = 1.0;

    /* cyclic Jacobi: rotate away each off-diagonal entry in turn */
    double total = 0.0;
    for (size_t i = 0; i < (size_t)d * d; ++i) total += C[i] * C[i];
    int sweep;
    for (sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int32_t p = 0; p < d; ++p)
            for (int32_t q = p + 1; q < d; ++q) off += C[(size_t)p * d + q] * C[(size_t)p * d + q];
        if (off <= 1e-32 * total || off == 0.0) break;
        for (int32_t p = 0; p < d; ++p) {
            for (int32_t q = p + 1; q < d; ++q) {
                double apq = C[(size_t)p * d + q];
                if (apq == 0.0) continue;
                double app = C[(size_t)p * d + p], aqq = C[(size_t)q * d + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = 1.0 / (fabs(theta) + sqrt(theta * theta + 1.0));
                if (theta < 0.0) t = -t;
                double c = 1.0 / sqrt(t * t + 1.0);
                double s = t * c;
                for (int32_t r = 0; r < d; ++r) {
                    if (r == p || r == q) continue;
                    double arp = C[(size_t)r * d + p], arq = C[(size_t)r * d + q];
                    double nrp = c * arp - s * arq;
                    double nrq = s * arp + c * arq;
                    C[(size_t)r * d + p] = nrp; C[(size_t)p * d + r] = nrp;
                    C[(size_t)r * d + q] = nrq; C[(size_t)q * d + r] = nrq;
                }
                C[(size_t)p * d + p] = app - t * apq;
                C[(size_t)q * d + q] = aqq + t * apq;
                C[(size_t)p * d + q] = 0.0;
                C[(size_t)q * d + p] = 0.0;
                for (int32_t r = 0; r < d; ++r) {
                    double erp = E[(size_t)r * d + p], erq = E[(size_t)r * d + q];
                    E[(size_t)r * d + p] = c * erp - s * erq;
                    E[(size_t)r * d + q] = s * erp + c * erq;
                }
            }
        }
    }
    int converged = sweep < 100;

    /* pick the k largest eigenvalues (selection, ties by lower index) */
    char* used = (char*)calloc((size_t)d, 1);
    for (int32_t c = 0; c < k; ++c) {
        int32_t best = -1;
        for (int32_t j = 0; j < d; ++j)
            if (!used[j] && (best < 0 || C[(size_t)j * d + j] > C[(size_t)best * d + best])) best = j;
        if (best < 0) break;
        used[best] = 1;
        lambda[c] = C[(size_t)best * d + best];
        int32_t arg = 0;
        for (int32_t r = 1; r < d; ++r)
            if (fabs(E[(size_t)r * d + best]) > fabs(E[(size_t)arg * d + best])) arg = r;
        double sg = E[(size_t)arg * d + best] < 0.0 ? -1.0 : 1.0;
        for (int32_t r = 0; r < d; ++r) V[(size_t)c * d + r] = sg * E[(size_t)r * d + best];
    }
    free(used); free(C); free(E);
    return converged ? sweep : -1;
}

/* --------------------------------------------------------------- cover -- */

void oracle_range(const double* f, int64_t n, int32_t m, int32_t j, double* lo, double* hi)
{
    double a = f[j], b = f[j];
    for (int64_t p = 1; p < n; ++p) {
        double v = f[p * m + j];
        if (v < a) a = v;
        if (v > b) b = v;
    }
    *lo = a; *hi = b;
}

/* n uniform intervals with overlap fraction p covering [lo, hi] (§3:
 * "the number of cover elements n and their percentage of overlaps p";
 * "Each interval (cover element) typically has uniform size"). */
void oracle_interval_bounds(double lo, double hi, int32_t n_int, double p, double* a, double* b)
{
    double span = hi - lo;
    double denom = (double)n_int - (double)(n_int - 1) * p;
    double L = (span == 0.0) ? 1.0 : span / denom;
    double s = L * (1.0 - p);
    for (int32_t k = 0; k < n_int; ++k) {
        a[k] = lo + (double)k * s;
        b[k] = a[k] + L;
    }
    a[0] = lo;
    b[n_int - 1] = hi;
    for (int32_t k = 0; k + 1 < n_int; ++k)
        if (b[k] < a[k + 1]) b[k] = a[k + 1];
}

static int cmp_double(const void* x, const void* y)
{
    const double a = *(const double*)x, b = *(const double*)y;
    return (a > b) - (a < b);
}

/* Balanced cover of one filter dimension (§3: some libraries offer a
 * "balanced" cover whose intervals hold equal numbers of points). Reading:
 * the uniform cover of the filter's ranks. With v_0 <= ... <= v_{n-1} the
 * sorted values, the uniform intervals [r_a, r_b] of n_int elements with
 * overlap p over the rank range [0, n-1] give the value intervals
 * [v_ceil(r_a), v_min(floor(r_b), n-1)]; one starting past the last rank is
 * empty (a = +inf). Membership stays closed, so an interval with
 * ceil(r_a) > floor(r_b) holds only points of a value tied at both ends.
 * The bounds are nondecreasing in k. */
void oracle_balanced_bounds(const double* lens, int64_t n, int32_t m, int32_t j, int32_t n_int, double p,
                            double* a, double* b)
{
    double* v = (double*)malloc(sizeof(double) * (size_t)n);
    for (int64_t q = 0; q < n; ++q) v[q] = lens[q * m + j];
    qsort(v, (size_t)n, sizeof(double), cmp_double);
    double* ra = (double*)malloc(sizeof(double) * (size_t)n_int);
    double* rb = (double*)malloc(sizeof(double) * (size_t)n_int);
    oracle_interval_bounds(0.0, (double)(n - 1), n_int, p, ra, rb);
    for (int32_t k = 0; k < n_int; ++k) {
        double lo_r = ceil(ra[k]), hi_r = floor(rb[k]);
        if (hi_r > (double)(n - 1)) hi_r = (double)(n - 1);
        b[k] = v[(int64_t)hi_r];
        a[k] = lo_r > (double)(n - 1) ? INFINITY : v[(int64_t)lo_r];
    }
    free(ra);
    free(rb);
    free(v);
}

/* Pull-back cover (§3: points in f^{-1}(V_k)). lens is n x m row-major.
 * Writes elem_offsets[E+1] and, when elem_points != NULL, the member
 * indices of each element in ascending order. Returns the total number of
 * memberships, or -1 on bad arguments. Brute force: every point is tested
 * against every element. */
int64_t oracle_cover(const double* lens, int64_t n, int32_t m, const int32_t* n_int,
                     const double* overlap, int32_t balanced, int64_t* elem_offsets, int32_t* elem_points)
{
    if (m < 1 || m > 2) return -1;
    double* a[2] = {0, 0};
    double* b[2] = {0, 0};
    for (int32_t j = 0; j < m; ++j) {
        double lo, hi;
        oracle_range(lens, n, m, j, &lo, &hi);
        a[j] = (double*)malloc(sizeof(double) * (size_t)n_int[j]);
        b[j] = (double*)malloc(sizeof(double) * (size_t)n_int[j]);
        if (balanced)
            oracle_balanced_bounds(lens, n, m, j, n_int[j], overlap[j], a[j], b[j]);
        else
            oracle_interval_bounds(lo, hi, n_int[j], overlap[j], a[j], b[j]);
    }
    int32_t n2 = (m == 2) ? n_int[1] : 1;
    int64_t E = (int64_t)n_int[0] * n2;
    int64_t total = 0;
    for (int64_t e = 0; e < E; ++e) {
        int32_t i = (int32_t)(e / n2), jj = (int32_t)(e % n2);
        elem_offsets[e] = total;
        for (int64_t p = 0; p < n; ++p) {
            double f0 = lens[p * m];
            int in = (a[0][i] <= f0) && (f0 <= b[0][i]);
            if (m == 2) {
                double f1 = lens[p * m + 1];
                in = in && (a[1][jj] <= f1) && (f1 <= b[1][jj]);
            }
            if (in) {
                if (elem_points) elem_points[total] = (int32_t)p;
                ++total;
            }
        }
    }
    elem_offsets[E] = total;
    for (int32_t j = 0; j < m; ++j) { free(a[j]); free(b[j]); }
    return total;
}

/* -------------------------------------------------------------- DBSCAN -- */

static double sqdist(const float* x, const float* y, int32_t d)
{
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double t = (double)x[k] - (double)y[k];
        s = s + t * t;
    }
    return s;
}

/* DBSCAN (§3: "eps is the neighborhood size of a given point, and minPts
 * is the minimum number of points needed to consider a collection of points
 * as a cluster"; Ester et al. 1996) on the points pts[0..np) of one cover
 * element, pts ascending.
 * Outputs per member i: count[i] = |N(pts[i])|, core[i], label[i] =
 * canonical cluster id (smallest global index of the cluster's core points)
 * or -1 for noise. *near_ties = number of unordered member pairs whose
 * squared distance lies within 1e-12 * eps^2 of eps^2. Returns 0. */
int oracle_dbscan(const float* X, int64_t n, int32_t d, int64_t ld,
                  const int32_t* pts, int64_t np, double eps, int32_t min_pts,
                  int32_t* count, uint8_t* core, int64_t* label, int64_t* near_ties)
{
    (void)n;
    const double eps2 = eps * eps;
    const double tie = 1e-12 * eps2;
    int64_t ties = 0;

    /* neighbour counts, self included */
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : ties)
    for (int64_t i = 0; i < np; ++i) {
        const float* xi = X + (int64_t)pts[i] * ld;
        int32_t c = 0;
        for (int64_t j = 0; j < np; ++j) {
            double s = sqdist(xi, X + (int64_t)pts[j] * ld, d);
            if (s <= eps2) ++c;
            if (j > i && fabs(s - eps2) <= tie) ++ties;
        }
        count[i] = c;
        core[i] = (uint8_t)(c >= min_pts);
    }
    *near_ties = ties;

    /* clusters: breadth-first search over core points, started from the
     * unvisited core of smallest index, so the start is the canonical id */
    for (int64_t i = 0; i < np; ++i) label[i] = -1;
    int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));
    for (int64_t s0 = 0; s0 < np; ++s0) {
        if (!core[s0] || label[s0] >= 0) continue;
        int64_t canon = pts[s0];
        int64_t head = 0, tail = 0;
        queue[tail++] = s0;
        label[s0] = canon;
        while (head < tail) {
            int64_t u = queue[head++];
            const float* xu = X + (int64_t)pts[u] * ld;
#pragma omp parallel for schedule(static)
            for (int64_t v = 0; v < np; ++v) {
                if (!core[v] || label[v] >= 0) continue;
                if (sqdist(xu, X + (int64_t)pts[v] * ld, d) <= eps2) label[v] = -2; /* mark */
            }
            for (int64_t v = 0; v < np; ++v)
                if (label[v] == -2) { label[v] = canon; queue[tail++] = v; }
        }
    }
    free(queue);

    /* border points: the neighbouring cluster of smallest canonical id */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < np; ++i) {
        if (core[i]) continue;
        const float* xi = X + (int64_t)pts[i] * ld;
        int64_t best = -1;
        for (int64_t j = 0; j < np; ++j) {
            if (!core[j]) continue;
            if (sqdist(xi, X + (int64_t)pts[j] * ld, d) <= eps2) {
                if (best < 0 || label[j] < best) best = label[j];
            }
        }
        label[i] = best;
    }
    return 0;
}

/* k-th nearest-neighbour distance (§5, "Visualizing Class Separation via
 * Neuron Activations": a module plots the distribution of the distances to
 * the k-th nearest neighbours, k = 5, to choose eps for DBSCAN). Reading:
 * for each query point p, the k-th smallest of the distances d(p, y) over all
 * points y of the cloud, p itself included (distance 0), so that p is a core
 * point of DBSCAN(eps, k) on the whole cloud iff kdist(p) <= eps. Distances
 * as in DBSCAN: the double sum of squared differences, k ascending, then
 * sqrt. Brute force: all n squared distances, sorted. Returns -1 for k
 * outside [1, n] or a query index outside [0, n). */
int oracle_knn_distance(const float* X, int64_t n, int32_t d, int64_t ld, const int32_t* queries, int64_t q,
                        int32_t k, double* out)
{
    if (k < 1 || k > n) return -1;
    int bad = 0;
#pragma omp parallel
    {
        double* d2 = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < q; ++i) {
            if (queries[i] < 0 || queries[i] >= n) { bad = 1; continue; }
            const float* x = X + (int64_t)queries[i] * ld;
            for (int64_t y = 0; y < n; ++y) d2[y] = sqdist(x, X + y * ld, d);
            qsort(d2, (size_t)n, sizeof(double), cmp_double);
            out[i] = sqrt(d2[k - 1]);
        }
        free(d2);
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------ single linkage -- */

/* Single-linkage clustering (§5: Lum et al. cluster each cover element by
 * single linkage, where this tool uses DBSCAN) is the minimum spanning tree
 * of the element's points: cutting it at a height h gives the clusters.
 * Reading: within one cover element (pts ascending, global indices), the
 * minimum spanning forest of the eps-graph, whose edges are the pairs with
 * squared distance d2 <= eps * eps (the DBSCAN distance above), ordered by
 * the key (d2, smaller point index, larger point index) so that the forest
 * is unique when distances tie: Kruskal's algorithm, i.e. every pair in key
 * order, kept iff its points are not joined yet (union-find). Writes the
 * kept edges in key order: u[k] < v[k] (global indices) and d2[k]; returns
 * their number (at most np - 1), or -1 if memory runs out. */
typedef struct {
    double d2;
    int32_t lo, hi;
} ms_edge;

static int cmp_edge(const void* x, const void* y)
{
    const ms_edge* a = (const ms_edge*)x;
    const ms_edge* b = (const ms_edge*)y;
    if (a->d2 != b->d2) return a->d2 < b->d2 ? -1 : 1;
    if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
    if (a->hi != b->hi) return a->hi < b->hi ? -1 : 1;
    return 0;
}

static int64_t uf_find(int64_t* parent, int64_t x)
{
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

int64_t oracle_msf(const float* X, int64_t n, int32_t d, int64_t ld, const int32_t* pts, int64_t np, double eps,
                   int32_t* u, int32_t* v, double* d2)
{
    (void)n;
    const double eps2 = eps * eps;
    /* every pair within eps, in member order */
    int64_t cap = 1024, m = 0;
    ms_edge* e = (ms_edge*)malloc(sizeof(ms_edge) * (size_t)cap);
    if (!e) return -1;
    for (int64_t i = 0; i < np; ++i) {
        const float* xi = X + (int64_t)pts[i] * ld;
        for (int64_t j = i + 1; j < np; ++j) {
            const double s = sqdist(xi, X + (int64_t)pts[j] * ld, d);
            if (s > eps2) continue;
            if (m == cap) {
                cap *= 2;
                ms_edge* t = (ms_edge*)realloc(e, sizeof(ms_edge) * (size_t)cap);
                if (!t) { free(e); return -1; }
                e = t;
            }
            e[m].d2 = s;
            e[m].lo = pts[i];
            e[m].hi = pts[j];
            ++m;
        }
    }
    qsort(e, (size_t)m, sizeof(ms_edge), cmp_edge);
    /* Kruskal: members are found by binary search in pts (ascending) */
    int64_t* parent = (int64_t*)malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));
    if (!parent) { free(e); return -1; }
    for (int64_t i = 0; i < np; ++i) parent[i] = i;
    int64_t kept = 0;
    for (int64_t k = 0; k < m && kept + 1 < np; ++k) {
        int64_t ia = 0, ib = 0;
        {
            int64_t lo = 0, hi = np - 1;
            while (lo < hi) { int64_t mid = (lo + hi) / 2; if (pts[mid] < e[k].lo) lo = mid + 1; else hi = mid; }
            ia = lo;
            lo = 0; hi = np - 1;
            while (lo < hi) { int64_t mid = (lo + hi) / 2; if (pts[mid] < e[k].hi) lo = mid + 1; else hi = mid; }
            ib = lo;
        }
        const int64_t ra = uf_find(parent, ia), rb = uf_find(parent, ib);
        if (ra == rb) continue;
        parent[ra < rb ? rb : ra] = ra < rb ? ra : rb;
        u[kept] = e[k].lo;
        v[kept] = e[k].hi;
        d2[kept] = e[k].d2;
        ++kept;
    }
    free(parent);
    free(e);
    return kept;
}
