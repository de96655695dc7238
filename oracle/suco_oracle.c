/*
 * suco_oracle.c -- CPU oracle for the SuCo query path (TEST INFRASTRUCTURE).
 *
 * This file is test infrastructure, not product code.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * It restates, slowly and literally, what the paper's method computes:
 *   - Definition 3 (subspace sampling), in the contiguous special case that
 *     Section 3.2 describes for SC-Linear: subspace i covers dims
 *     [i*s, (i+1)*s) with s = floor(d/Ns); the last subspace takes the rest.
 *   - Algorithm 2 (Create Index): per subspace, two half-subspace K-means
 *     codebooks of sqrt(K) centroids and an inverted multi-index (IMI) that maps
 *     the cell (a1, a2) to the ids assigned to it.
 *   - Algorithm 3 (Dynamic Activation): the literal heap-free walk over the
 *     sorted half-subspace distance lists.
 *   - Algorithm 4 (k-ANN Query): SC-score counting (Definition 4), selection of
 *     the beta*n highest scores, exact re-rank, top-k.
 *   - Algorithm 1 (SC-Linear) and exact k-NN by brute force, as cross-checks.
 *
 * Arithmetic is double precision (FP64) everywhere except where a floating
 * point value decides a discrete outcome that the GPU path also decides: the
 * cell ranking of Algorithm 3.  There the oracle can take the decision in the
 * GPU kernel's precision (rank_precision = 1): each half-subspace squared
 * distance is accumulated in FP32 as acc = fmaf(q_j - c_j, q_j - c_j, acc)
 * over j in ascending order, and the cell sum d1 + d2 is one FP32 addition.
 * This file must be compiled with -ffp-contract=off so that no other
 * expression is fused.
 *
 * Readings of passages the paper leaves open (each one is listed in the
 * design notes as well):
 *   R1  distances inside Algorithms 3/4 are squared Euclidean distances; the
 *       cell value is d1[a1] + d2[a2], the squared distance to the product
 *       centroid.
 *   R2  Algorithm 3 never retires a row whose last column was retrieved; here
 *       such a row's active distance becomes +infinity.  Rows not yet
 *       activated also hold +infinity.
 *   R3  "index of the minimum element" is the first (lowest) such index.
 *   R4  T = ceil(alpha*n - 1e-9) clamped to [1, n] (Algorithm 3 stops once the
 *       retrieved count reaches alpha*n); C = ceil(beta*n - 1e-9) raised to at
 *       least k and clamped to [1, n].
 *   R5  argsort of the centroid distances is stable (ties by centroid index).
 *   R6  candidates are the first C ids when sorted by (score desc, id asc);
 *       results are sorted by (distance asc, id asc); missing results are
 *       padded with id -1 and distance +infinity.
 *   R7  K-means (not specified in the paper): Lloyd iterations from the given
 *       initial ids; an empty cluster keeps its previous centroid; argmin ties
 *       go to the lowest centroid index; the index stores FP32 centroids and the
 *       final assignment is taken against those stored centroids.
 *   R8  the IMI cell id of (a1, a2) is a1*sqrtK + a2; ids inside a cell are in
 *       ascending order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Subspace layout: Definition 3, contiguous case (Section 3.2); halves as in
 * Algorithm 2 (first floor(len/2) dims, then the rest).                     */

ORC_EXPORT void orc_subspace_dims(int32_t d, int32_t Ns, int32_t i, int32_t* off, int32_t* len)
{
    int32_t s = d / Ns;
    *off = i * s;
    *len = (i == Ns - 1) ? d - (Ns - 1) * s : s;
}

ORC_EXPORT void orc_half_dims(int32_t d, int32_t Ns, int32_t i, int32_t h, int32_t* off, int32_t* len)
{
    int32_t so, sl;
    orc_subspace_dims(d, Ns, i, &so, &sl);
    int32_t first = sl / 2;
    if (h == 0) {
        *off = so;
        *len = first;
    } else {
        *off = so + first;
        *len = sl - first;
    }
}

/* Largest half length: the second half of the last (largest) subspace. */
ORC_EXPORT int32_t orc_hmax(int32_t d, int32_t Ns)
{
    int32_t off, len;
    orc_half_dims(d, Ns, Ns - 1, 1, &off, &len);
    return len;
}

/* ------------------------------------------------------------------------ */
/* Reading R4: the integer thresholds.                                       */

ORC_EXPORT int64_t orc_collision_threshold(double alpha, int64_t n)
{
    double t = ceil(alpha * (double)n - 1e-9);
    if (t < 1.0) t = 1.0;
    if (t > (double)n) t = (double)n;
    return (int64_t)t;
}

ORC_EXPORT int64_t orc_candidate_count(double beta, int64_t n, int32_t k)
{
    double c = ceil(beta * (double)n - 1e-9);
    if (c < (double)k) c = (double)k;
    if (c > (double)n) c = (double)n;
    if (c < 1.0) c = 1.0;
    return (int64_t)c;
}

/* ------------------------------------------------------------------------ */
/* Distances                                                                 */

/* The distance between two vectors of length len, FP64.  metric 0: squared
 * Euclidean (the paper's default); metric 1: Manhattan (L1), the variant of
 * Section 5's distance-measure experiment (SuCo-L1).  Both are sums of
 * per-dimension terms, so a cell's value d1 + d2 is the distance to its
 * product centroid in either metric. */
static double dist64(const float* a, const float* b, int32_t len, int32_t metric)
{
    double acc = 0.0;
    for (int32_t j = 0; j < len; ++j) {
        double t = (double)a[j] - (double)b[j];
        acc += metric == 1 ? fabs(t) : t * t;
    }
    return acc;
}

/* Same, FP32 in ascending dimension order: acc = fmaf(t, t, acc) for the
 * squared Euclidean distance, acc = acc + |t| for L1 (t = a_j - b_j). */
static float dist32(const float* a, const float* b, int32_t len, int32_t metric)
{
    float acc = 0.0f;
    for (int32_t j = 0; j < len; ++j) {
        float t = a[j] - b[j];
        acc = metric == 1 ? acc + fabsf(t) : fmaf(t, t, acc);
    }
    return acc;
}

/* ------------------------------------------------------------------------ */
/* Reading R5: stable argsort by insertion (sqrt(K) <= 256, so O(m^2) is fine). */

ORC_EXPORT void orc_argsort_stable(const double* v, int32_t m, int32_t* idx)
{
    for (int32_t i = 0; i < m; ++i) idx[i] = i;
    for (int32_t i = 1; i < m; ++i) {
        int32_t cur = idx[i];
        int32_t j = i - 1;
        while (j >= 0 && v[idx[j]] > v[cur]) {
            idx[j + 1] = idx[j];
            --j;
        }
        idx[j + 1] = cur;
    }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 3: Dynamic Activation, literally, with readings R2 and R3.
 *
 * dists1/dists2: distances of the query half to each centroid (length sqrtK).
 * idx1/idx2:     their stable ascending argsorts.
 * cell_size:     ids per IMI cell, indexed by a1*sqrtK + a2.
 * precision:     0 = cell sum in FP64, 1 = cell sum as one FP32 addition of the
 *                (FP32-valued) distances.
 * out_cells:     retrieved cell ids in retrieval order (capacity sqrtK^2).
 * trace_rows:    optional; after the r-th retrieval, the number of activated
 *                rows of dists1 (capacity sqrtK^2).
 * Returns the number of retrieved cells; *retrieved_num gets the id count. */

static double cell_sum(const double* d1, const double* d2, int32_t a1, int32_t a2, int32_t precision)
{
    if (precision == 1) {
        float s = (float)d1[a1] + (float)d2[a2];
        return (double)s;
    }
    return d1[a1] + d2[a2];
}

ORC_EXPORT int64_t orc_dynamic_activation(int64_t T, int32_t sqrtK, const double* dists1, const int32_t* idx1,
                                          const double* dists2, const int32_t* idx2, const int64_t* cell_size,
                                          int32_t precision, int32_t* out_cells, int64_t* retrieved_num,
                                          int32_t* trace_rows)
{
    int32_t* active_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)sqrtK);
    double* active_dists = (double*)malloc(sizeof(double) * (size_t)sqrtK);
    for (int32_t r = 0; r < sqrtK; ++r) {
        active_idx[r] = -1;
        active_dists[r] = INFINITY;
    }
    int64_t retrieved = 0;
    int64_t ncells = 0;
    int32_t rows_active = 1;
    active_idx[0] = 0;
    active_dists[0] = cell_sum(dists1, dists2, idx1[0], idx2[0], precision);
    for (;;) {
        /* the first minimum of active_dists (R3) */
        int32_t pos = -1;
        double best = INFINITY;
        for (int32_t r = 0; r < sqrtK; ++r) {
            if (active_dists[r] < best) {
                best = active_dists[r];
                pos = r;
            }
        }
        if (pos < 0) break; /* every cell retrieved (only if T > n) */
        int32_t cell = idx1[pos] * sqrtK + idx2[active_idx[pos]];
        out_cells[ncells++] = cell;
        retrieved += cell_size[cell];
        if (retrieved >= T) {
            if (trace_rows) trace_rows[ncells - 1] = rows_active;
            break;
        }
        if (active_idx[pos] == 0 && pos < sqrtK - 1) {
            active_idx[pos + 1] = 0;
            active_dists[pos + 1] = cell_sum(dists1, dists2, idx1[pos + 1], idx2[0], precision);
            rows_active++;
        }
        if (active_idx[pos] < sqrtK - 1) {
            active_idx[pos]++;
            active_dists[pos] = cell_sum(dists1, dists2, idx1[pos], idx2[active_idx[pos]], precision);
        } else {
            active_dists[pos] = INFINITY; /* R2: the row is exhausted */
        }
        if (trace_rows) trace_rows[ncells - 1] = rows_active;
    }
    free(active_idx);
    free(active_dists);
    *retrieved_num = retrieved;
    return ncells;
}

/* ------------------------------------------------------------------------ */
/* Candidate selection (Algorithm 4, last loop; R6) and exact re-rank.       */

typedef struct {
    int32_t score;
    int64_t id;
} scored_t;

static int cmp_scored(const void* a, const void* b)
{
    const scored_t* x = (const scored_t*)a;
    const scored_t* y = (const scored_t*)b;
    if (x->score != y->score) return (x->score > y->score) ? -1 : 1;
    return (x->id < y->id) ? -1 : (x->id > y->id);
}

typedef struct {
    double dist;
    int64_t id;
} hit_t;

static int cmp_hit(const void* a, const void* b)
{
    const hit_t* x = (const hit_t*)a;
    const hit_t* y = (const hit_t*)b;
    if (x->dist != y->dist) return (x->dist < y->dist) ? -1 : 1;
    return (x->id < y->id) ? -1 : (x->id > y->id);
}

/* The first C ids by (score desc, id asc). */
ORC_EXPORT void orc_select_candidates(const int32_t* scores, int64_t n, int64_t C, int64_t* out_cands)
{
    scored_t* s = (scored_t*)malloc(sizeof(scored_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        s[i].score = scores[i];
        s[i].id = i;
    }
    qsort(s, (size_t)n, sizeof(scored_t), cmp_scored);
    for (int64_t z = 0; z < C; ++z) out_cands[z] = s[z].id;
    free(s);
}

/* Exact squared distances from q to the listed rows, sorted by (dist, id);
 * the first k go out, padded with (-1, +inf). */
ORC_EXPORT void orc_rerank(const float* X, int32_t d, const float* q, const int64_t* ids, int64_t m, int32_t k,
                           int64_t* out_ids, double* out_dist, int32_t metric)
{
    hit_t* h = (hit_t*)malloc(sizeof(hit_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t z = 0; z < m; ++z) {
        h[z].id = ids[z];
        h[z].dist = dist64(X + (size_t)ids[z] * (size_t)d, q, d, metric);
    }
    qsort(h, (size_t)m, sizeof(hit_t), cmp_hit);
    for (int32_t z = 0; z < k; ++z) {
        if (z < m) {
            out_ids[z] = h[z].id;
            out_dist[z] = h[z].dist;
        } else {
            out_ids[z] = -1;
            out_dist[z] = INFINITY;
        }
    }
    free(h);
}

/* Exact k-NN over the whole dataset (the recall reference of Section 5.1). */
ORC_EXPORT void orc_bruteforce_knn(const float* X, int64_t n, int32_t d, const float* q, int32_t k,
                                   int64_t* out_ids, double* out_dist, int32_t metric)
{
    int64_t* all = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) all[i] = i;
    orc_rerank(X, d, q, all, n, k, out_ids, out_dist, metric);
    free(all);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: K-means per half-subspace, then the IMI.                     */

/* Lloyd's algorithm on dims [off, off+len) of X (row stride d).
 * cent: k*len doubles out.  assign: n ints out (assignment from the last
 * assignment step, i.e. against the centroids before the last update).     */
ORC_EXPORT void orc_kmeans(const float* X, int64_t n, int32_t d, int32_t off, int32_t len, int32_t k,
                           int32_t iters, const int64_t* init_ids, double* cent, int32_t* assign, int32_t metric)
{
    for (int32_t a = 0; a < k; ++a)
        for (int32_t j = 0; j < len; ++j) cent[(size_t)a * len + j] = (double)X[(size_t)init_ids[a] * d + off + j];
    double* sum = (double*)malloc(sizeof(double) * (size_t)k * (size_t)len);
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
    for (int32_t it = 0; it < iters; ++it) {
        /* assignment step: nearest centroid, ties to the lowest index */
        for (int64_t p = 0; p < n; ++p) {
            const float* x = X + (size_t)p * d + off;
            int32_t best = 0;
            double bd = INFINITY;
            for (int32_t a = 0; a < k; ++a) {
                double acc = 0.0;
                for (int32_t j = 0; j < len; ++j) {
                    double t = (double)x[j] - cent[(size_t)a * len + j];
                    acc += metric == 1 ? fabs(t) : t * t;
                }
                if (acc < bd) {
                    bd = acc;
                    best = a;
                }
            }
            assign[p] = best;
        }
        /* update step: mean of the members; an empty cluster keeps its centroid */
        memset(sum, 0, sizeof(double) * (size_t)k * (size_t)len);
        memset(cnt, 0, sizeof(int64_t) * (size_t)k);
        for (int64_t p = 0; p < n; ++p) {
            const float* x = X + (size_t)p * d + off;
            int32_t a = assign[p];
            cnt[a]++;
            for (int32_t j = 0; j < len; ++j) sum[(size_t)a * len + j] += (double)x[j];
        }
        for (int32_t a = 0; a < k; ++a)
            if (cnt[a] > 0)
                for (int32_t j = 0; j < len; ++j) cent[(size_t)a * len + j] = sum[(size_t)a * len + j] / (double)cnt[a];
    }
    free(sum);
    free(cnt);
}

/* Nearest stored (FP32) centroid of each point, FP64 distances, ties low. */
ORC_EXPORT void orc_assign_nearest(const float* X, int64_t n, int32_t d, int32_t off, int32_t len, const float* cent,
                                   int32_t k, int32_t cent_stride, int32_t* assign, int32_t metric)
{
    for (int64_t p = 0; p < n; ++p) {
        int32_t best = 0;
        double bd = INFINITY;
        for (int32_t a = 0; a < k; ++a) {
            double acc = dist64(X + (size_t)p * d + off, cent + (size_t)a * cent_stride, len, metric);
            if (acc < bd) {
                bd = acc;
                best = a;
            }
        }
        assign[p] = best;
    }
}

/* IMI of one subspace (Algorithm 2, inner loop; R8): cell_off has K+1
 * entries, perm lists the ids of each cell in ascending order. */
ORC_EXPORT void orc_imi_from_assign(const int32_t* assign1, const int32_t* assign2, int64_t n, int32_t sqrtK,
                                    int64_t* cell_off, int64_t* perm)
{
    int64_t K = (int64_t)sqrtK * sqrtK;
    for (int64_t c = 0; c <= K; ++c) cell_off[c] = 0;
    for (int64_t p = 0; p < n; ++p) cell_off[(int64_t)assign1[p] * sqrtK + assign2[p] + 1]++;
    for (int64_t c = 0; c < K; ++c) cell_off[c + 1] += cell_off[c];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)K);
    for (int64_t c = 0; c < K; ++c) fill[c] = cell_off[c];
    for (int64_t p = 0; p < n; ++p) {
        int64_t c = (int64_t)assign1[p] * sqrtK + assign2[p];
        perm[fill[c]++] = p;
    }
    free(fill);
}

/* Algorithm 2 in full.  centroids: [Ns][2][sqrtK][hmax] floats out (zero
 * padded); assign: [Ns][2][n] out; cell_off: [Ns][K+1]; perm: [Ns][n].
 * init_ids: [Ns][2][sqrtK] point ids that seed Lloyd's iterations. */
ORC_EXPORT void orc_build_index(const float* X, int64_t n, int32_t d, int32_t Ns, int32_t sqrtK, int32_t iters,
                                const int64_t* init_ids, float* centroids, int32_t* assign, int64_t* cell_off,
                                int64_t* perm, int32_t nthreads, int32_t metric)
{
    int32_t hmax = orc_hmax(d, Ns);
    int64_t K = (int64_t)sqrtK * sqrtK;
    memset(centroids, 0, sizeof(float) * (size_t)Ns * 2 * sqrtK * hmax);
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int32_t ih = 0; ih < 2 * Ns; ++ih) {
        int32_t i = ih / 2, h = ih % 2, off, len;
        orc_half_dims(d, Ns, i, h, &off, &len);
        double* cent = (double*)malloc(sizeof(double) * (size_t)sqrtK * len);
        int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        orc_kmeans(X, n, d, off, len, sqrtK, iters, init_ids + (size_t)ih * sqrtK, cent, tmp, metric);
        float* cf = centroids + (size_t)ih * sqrtK * hmax;
        for (int32_t a = 0; a < sqrtK; ++a)
            for (int32_t j = 0; j < len; ++j) cf[(size_t)a * hmax + j] = (float)cent[(size_t)a * len + j];
        orc_assign_nearest(X, n, d, off, len, cf, sqrtK, hmax, assign + (size_t)ih * n, metric);
        free(cent);
        free(tmp);
    }
    for (int32_t i = 0; i < Ns; ++i)
        orc_imi_from_assign(assign + (size_t)(2 * i) * n, assign + (size_t)(2 * i + 1) * n, n, sqrtK,
                            cell_off + (size_t)i * (K + 1), perm + (size_t)i * n);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 4: k-ANN query for one query q.
 *
 * rank_precision: 0 = FP64 centroid distances and cell sums (the paper's
 * arithmetic), 1 = the GPU kernel's FP32 decision arithmetic (see header).
 * Optional outputs (NULL to skip): scores [n]; cands [C]; teff [Ns] (ids
 * collided per subspace); activated [Ns][K] (1 = cell retrieved);
 * dtab [Ns][2][sqrtK] (the centroid distances as used for ranking). */
/* Algorithm 4 for one query.  dtab_in (nullable, [Ns][2][sqrtK]) supplies the
 * half-subspace centroid distances instead of computing them (the tables of
 * a reduced-precision ranking); everything after them is unchanged. */
static int query_core(const float* X, int64_t n, int32_t d, int32_t Ns, int32_t sqrtK, const float* centroids,
                      const int64_t* cell_off, const int64_t* perm, const float* q, int32_t k, int64_t T, int64_t C,
                      int32_t rank_precision, const double* dtab_in, int64_t* out_ids, double* out_dist,
                      int32_t* scores_out, int64_t* cands_out, int64_t* teff_out, uint8_t* activated_out,
                      double* dtab_out, int32_t metric)
{
    int32_t hmax = orc_hmax(d, Ns);
    int64_t K = (int64_t)sqrtK * sqrtK;
    int32_t* scores = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    double* dists1 = (double*)malloc(sizeof(double) * (size_t)sqrtK);
    double* dists2 = (double*)malloc(sizeof(double) * (size_t)sqrtK);
    int32_t* idx1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)sqrtK);
    int32_t* idx2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)sqrtK);
    int64_t* csize = (int64_t*)malloc(sizeof(int64_t) * (size_t)K);
    int32_t* cells = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
    if (activated_out) memset(activated_out, 0, (size_t)Ns * (size_t)K);
    for (int32_t i = 0; i < Ns; ++i) {
        for (int32_t h = 0; h < 2; ++h) {
            int32_t off, len;
            orc_half_dims(d, Ns, i, h, &off, &len);
            double* dd = h == 0 ? dists1 : dists2;
            const float* cb = centroids + (size_t)(2 * i + h) * sqrtK * hmax;
            for (int32_t a = 0; a < sqrtK; ++a) {
                if (dtab_in)
                    dd[a] = dtab_in[((size_t)i * 2 + h) * sqrtK + a];
                else if (rank_precision == 1)
                    dd[a] = (double)dist32(q + off, cb + (size_t)a * hmax, len, metric);
                else
                    dd[a] = dist64(q + off, cb + (size_t)a * hmax, len, metric);
            }
            if (dtab_out)
                for (int32_t a = 0; a < sqrtK; ++a) dtab_out[((size_t)i * 2 + h) * sqrtK + a] = dd[a];
        }
        orc_argsort_stable(dists1, sqrtK, idx1);
        orc_argsort_stable(dists2, sqrtK, idx2);
        const int64_t* co = cell_off + (size_t)i * (K + 1);
        for (int64_t c = 0; c < K; ++c) csize[c] = co[c + 1] - co[c];
        int64_t got = 0;
        int64_t nc = orc_dynamic_activation(T, sqrtK, dists1, idx1, dists2, idx2, csize, rank_precision, cells, &got,
                                            NULL);
        if (teff_out) teff_out[i] = got;
        /* every id of every retrieved cell collides: its SC-score grows by one */
        const int64_t* pm = perm + (size_t)i * n;
        for (int64_t z = 0; z < nc; ++z) {
            int32_t c = cells[z];
            if (activated_out) activated_out[(size_t)i * K + c] = 1;
            for (int64_t p = co[c]; p < co[c + 1]; ++p) scores[pm[p]] += 1;
        }
    }
    int64_t* cands = (int64_t*)malloc(sizeof(int64_t) * (size_t)C);
    orc_select_candidates(scores, n, C, cands);
    orc_rerank(X, d, q, cands, C, k, out_ids, out_dist, metric);
    if (scores_out) memcpy(scores_out, scores, sizeof(int32_t) * (size_t)n);
    if (cands_out) memcpy(cands_out, cands, sizeof(int64_t) * (size_t)C);
    free(cands);
    free(scores);
    free(dists1);
    free(dists2);
    free(idx1);
    free(idx2);
    free(csize);
    free(cells);
    return 0;
}

ORC_EXPORT int orc_query(const float* X, int64_t n, int32_t d, int32_t Ns, int32_t sqrtK, const float* centroids,
                         const int64_t* cell_off, const int64_t* perm, const float* q, int32_t k, int64_t T,
                         int64_t C, int32_t rank_precision, int64_t* out_ids, double* out_dist, int32_t* scores_out,
                         int64_t* cands_out, int64_t* teff_out, uint8_t* activated_out, double* dtab_out,
                         int32_t metric)
{
    return query_core(X, n, d, Ns, sqrtK, centroids, cell_off, perm, q, k, T, C, rank_precision, NULL, out_ids,
                      out_dist, scores_out, cands_out, teff_out, activated_out, dtab_out, metric);
}

/* Algorithm 4 for one query from given centroid-distance tables (the ranking
 * is then taken in FP32, as rank_precision 1). */
ORC_EXPORT int orc_query_from_tables(const float* X, int64_t n, int32_t d, int32_t Ns, int32_t sqrtK,
                                     const float* centroids, const int64_t* cell_off, const int64_t* perm,
                                     const float* q, int32_t k, int64_t T, int64_t C, const double* dtab_in,
                                     int64_t* out_ids, double* out_dist, int32_t* scores_out, int64_t* cands_out,
                                     int64_t* teff_out, uint8_t* activated_out, int32_t metric)
{
    return query_core(X, n, d, Ns, sqrtK, centroids, cell_off, perm, q, k, T, C, 1, dtab_in, out_ids, out_dist,
                      scores_out, cands_out, teff_out, activated_out, NULL, metric);
}

/* Algorithm 4 over a batch of nq queries, one query per OpenMP thread. */
ORC_EXPORT int orc_query_batch(const float* X, int64_t n, int32_t d, int32_t Ns, int32_t sqrtK, const float* centroids,
                               const int64_t* cell_off, const int64_t* perm, const float* Q, int64_t nq, int32_t k,
                               int64_t T, int64_t C, int32_t rank_precision, int32_t nthreads, int64_t* out_ids,
                               double* out_dist, int32_t metric)
{
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t b = 0; b < nq; ++b)
        orc_query(X, n, d, Ns, sqrtK, centroids, cell_off, perm, Q + (size_t)b * d, k, T, C, rank_precision,
                  out_ids + (size_t)b * k, out_dist + (size_t)b * k, NULL, NULL, NULL, NULL, NULL, metric);
    return 0;
}

/* The same with one (T, C) pair per query (per-query alpha and beta). */
ORC_EXPORT int orc_query_batch_pq(const float* X, int64_t n, int32_t d, int32_t Ns, int32_t sqrtK,
                                  const float* centroids, const int64_t* cell_off, const int64_t* perm, const float* Q,
                                  int64_t nq, int32_t k, const int64_t* T, const int64_t* C, int32_t rank_precision,
                                  int32_t nthreads, int64_t* out_ids, double* out_dist, int32_t metric)
{
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t b = 0; b < nq; ++b)
        orc_query(X, n, d, Ns, sqrtK, centroids, cell_off, perm, Q + (size_t)b * d, k, T[b], C[b], rank_precision,
                  out_ids + (size_t)b * k, out_dist + (size_t)b * k, NULL, NULL, NULL, NULL, NULL, metric);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: SC-Linear (no index).  Per subspace, the T points nearest to
 * q in that subspace (sorted by (distance, id)) collide.  precision 0 takes
 * the subspace distances in FP64, 1 in the GPU kernel's FP32 arithmetic
 * (acc = fmaf(x_j - q_j, x_j - q_j, acc) over the subspace's dims in order):
 * the collisions are a discrete decision that both sides must take in the
 * same precision.  Optional outputs: scores [n], cands [C].                  */

ORC_EXPORT int orc_sc_linear(const float* X, int64_t n, int32_t d, int32_t Ns, const float* q, int32_t k, int64_t T,
                             int64_t C, int32_t precision, int64_t* out_ids, double* out_dist, int32_t* scores_out,
                             int64_t* cands_out, int32_t metric)
{
    int32_t* scores = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    hit_t* h = (hit_t*)malloc(sizeof(hit_t) * (size_t)n);
    for (int32_t i = 0; i < Ns; ++i) {
        int32_t off, len;
        orc_subspace_dims(d, Ns, i, &off, &len);
        for (int64_t p = 0; p < n; ++p) {
            h[p].id = p;
            const float* x = X + (size_t)p * d + off;
            h[p].dist = precision == 1 ? (double)dist32(x, q + off, len, metric) : dist64(x, q + off, len, metric);
        }
        qsort(h, (size_t)n, sizeof(hit_t), cmp_hit);
        for (int64_t z = 0; z < T; ++z) scores[h[z].id] += 1;
    }
    int64_t* cands = (int64_t*)malloc(sizeof(int64_t) * (size_t)C);
    orc_select_candidates(scores, n, C, cands);
    orc_rerank(X, d, q, cands, C, k, out_ids, out_dist, metric);
    if (scores_out) memcpy(scores_out, scores, sizeof(int32_t) * (size_t)n);
    if (cands_out) memcpy(cands_out, cands, sizeof(int64_t) * (size_t)C);
    free(cands);
    free(h);
    free(scores);
    return 0;
}

ORC_EXPORT int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
