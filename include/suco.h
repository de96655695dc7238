/*
 * suco.h -- C ABI of the GB300 (sm_103a) SuCo library.
 *
 * SuCo answers approximate k-nearest-neighbour queries by subspace collision
 * (arXiv 2411.14754).  The dataset D holds n points in R^d (problem statement,
 * Section 1).  The index (Section 4.1, Algorithm 2) splits the d dimensions
 * into Ns contiguous subspaces (Definition 3, contiguous case of Section 3.2;
 * the last subspace takes the remainder), splits each subspace into two halves
 * (first floor(len/2) dims, then the rest), clusters each half with K-means
 * into sqrtK centroids, and keeps per subspace an inverted multi-index (IMI)
 * from each of the K = sqrtK^2 product cells to the ids that fall in it.
 * A query (Section 4.2, Algorithms 3 and 4) ranks the cells of every subspace
 * by the summed squared half-subspace centroid distance, collides the ids of
 * the best cells until alpha*n ids are reached, counts each id's SC-score
 * (Definition 4: the number of subspaces in which it collided), keeps the
 * beta*n best-scoring ids and returns the k nearest of them by exact squared
 * Euclidean distance.
 *
 * Conventions for every entry point:
 *   - Pointers marked (device) are CUDA device pointers on the current device;
 *     pointers marked (host) are host memory.  The caller owns every buffer it
 *     passes in; the library owns the index.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Device work
 *     is enqueued on it; unless stated otherwise the call returns as soon as
 *     the work is enqueued, and results are valid after the caller
 *     synchronises that stream.
 *   - Every call returns SUCO_OK (0) or a negative error code and never aborts
 *     the process; suco_last_error() returns a message for the calling
 *     thread's last failed call.
 *   - Thresholds: T = ceil(alpha*n - 1e-9) clamped to [1, n] ids collide per
 *     subspace (Algorithm 3 stops once alpha*n ids are retrieved; the last
 *     cell is taken whole, so T_eff >= T), and C = ceil(beta*n - 1e-9), raised
 *     to at least k and clamped to [1, n], candidates are re-ranked
 *     (Algorithm 4).
 *   - Ties: cells are ordered by (FP32 cell sum, rank of the first-half
 *     centroid, rank of the second-half centroid), which is the order in which
 *     Algorithm 3 retrieves them; candidates by (score desc, id asc); results
 *     by (squared distance asc, id asc).
 */
#ifndef SUCO_H
#define SUCO_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SUCO_API __attribute__((visibility("default")))
#else
#define SUCO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define SUCO_OK 0
#define SUCO_EINVAL (-1)       /* an argument is out of range or a pointer is NULL */
#define SUCO_ENOMEM (-2)       /* a device or host allocation failed              */
#define SUCO_ECUDA (-3)        /* a CUDA runtime call or a kernel launch failed   */
#define SUCO_ETIMEOUT (-4)     /* a bounded device-side wait gave up              */
#define SUCO_ESTATE (-5)       /* the index or the device is in the wrong state   */
#define SUCO_EUNSUPPORTED (-6) /* valid, but beyond this build's size limits      */

typedef struct suco_index suco_index; /* opaque; owned by the library */

/* Distance of an index (suco_build_params.metric).  L2: squared Euclidean,
 * the paper's default.  L1: Manhattan, the variant of Section 5's
 * distance-measure experiment (SuCo-L1): half-subspace centroid distances,
 * cell values d1 + d2 (L1 is a sum over dims, so this is the distance to the
 * product centroid), K-means assignments and the re-rank all use it, and
 * result distances are L1 distances.  An L1 index takes only FP32 ranking and
 * re-rank (the tensor-core and coarse forms are squared-L2 expansions) and
 * CTAs of 512 threads. */
#define SUCO_METRIC_L2 0
#define SUCO_METRIC_L1 1

/* Index construction parameters (Algorithm 2). */
typedef struct suco_build_params {
    int32_t Ns;              /* number of subspaces, 1..32                              */
    int32_t sqrtK;           /* centroids per half-subspace codebook, 1..256, <= n      */
    int32_t kmeans_iters;    /* Lloyd iterations t (0 keeps the initial points)        */
    int32_t metric;          /* SUCO_METRIC_L2 (0) or SUCO_METRIC_L1                   */
    uint64_t seed;           /* seeds the initial-centroid draw when init_ids is NULL  */
    const int64_t* init_ids; /* (host, nullable) [Ns][2][sqrtK] distinct point ids that
                                seed Lloyd's iterations, one list per half-subspace      */
    const int32_t* dim_perm; /* (host, nullable) Definition 3's subspace sampling: a
                                permutation of [0, d); subspace i < Ns-1 takes dims
                                dim_perm[i*s .. (i+1)*s) (s = floor(d/Ns)), the last the
                                rest, each half the first floor(len/2) of its list and
                                then the rest.  NULL: contiguous subspaces (Section 3.2).
                                The index stores D with its columns in this order, and
                                queries are read through it.                          */
} suco_build_params;

/* Builds the index of Algorithm 2 on the GPU: K-means per half-subspace
 * (sqrtK centroids, kmeans_iters Lloyd iterations from init_ids; an empty
 * cluster keeps its centroid; argmin ties go to the lowest centroid index),
 * then the IMI of each subspace (cell id a1*sqrtK + a2, ids ascending within a
 * cell).
 *   data  (device) n x d FP32, row-major.  Copied into the index; the caller
 *         may free it once the call returns.
 *   n     1 .. 2^31-1 points, with Ns*n < 2^32.   d  >= 2*Ns dimensions.
 *   out   receives the new index.  Synchronous: returns after the build ends.
 * Errors: SUCO_EINVAL on bad sizes or NULL pointers, SUCO_ENOMEM, SUCO_ECUDA. */
SUCO_API int suco_build_index(const float* data, int64_t n, int32_t d, const suco_build_params* params, void* stream,
                     suco_index** out);

/* Builds an index from given centroids and assignments instead of running
 * K-means (the IMI part of Algorithm 2 only).
 *   data       (device) n x d FP32 row-major, copied.
 *   centroids  (host) [Ns][2][sqrtK][hmax] FP32, hmax = ceil(len_last/2) where
 *              len_last = d - (Ns-1)*floor(d/Ns); entries past a half's length
 *              are ignored.
 *   assign     (host) [Ns][2][n] int32 centroid index of every point in every
 *              half-subspace, each in [0, sqrtK).
 * Synchronous.  Errors: as suco_build_index, and SUCO_EINVAL for an
 * assignment out of range. */
SUCO_API int suco_build_index_from_assignments(const float* data, int64_t n, int32_t d, int32_t Ns, int32_t sqrtK,
                                      const float* centroids, const int32_t* assign, void* stream,
                                      suco_index** out);

/* The IMI part of Algorithm 2 from given centroids and assignments, for any
 * metric and subspace sampling of `params` (Ns, sqrtK, metric, dim_perm;
 * kmeans_iters, seed and init_ids are ignored).
 *   centroids  (host) [Ns][2][sqrtK][hmax] FP32 over each half's dims in the
 *              sampling's order.   assign  (host) [Ns][2][n] int32 in [0, sqrtK).
 * Synchronous.  Errors: as suco_build_index_from_assignments. */
SUCO_API int suco_build_index_from_parts(const float* data, int64_t n, int32_t d, const suco_build_params* params,
                                         const float* centroids, const int32_t* assign, void* stream,
                                         suco_index** out);

/* Query parameters (Algorithm 4).  The three per-query arrays are optional;
 * a query without an array entry uses the scalar.  With per-query values the
 * thresholds are computed per query on the device by the same formula: T_b
 * from alpha_b, C_b from beta_b and k_b.  The scalar beta is an upper bound:
 * it sizes the candidate storage, and C_b never exceeds C(beta, k).  A
 * per-query k_b < k leaves result columns k_b..k-1 padded (-1, +inf). */
/* suco_query_params.flags: by default the grid holds as many clusters as fit
 * on the GPU at once and each cluster answers its share of the batch in turn;
 * this flag launches one cluster per query instead. */
#define SUCO_QUERY_ONE_CLUSTER_PER_QUERY 1

/* suco_query_params.precision: how the beta*n candidates are re-ranked.
 * FP32 computes every candidate's exact squared distance (Algorithm 4).
 * BF16 (not in the paper) first computes a coarse squared distance of every
 * candidate from the index's BF16 copy of D (values decoded exactly, sums in
 * FP32); the exact_rerank candidates with the smallest (coarse distance, id)
 * over the whole query survive, and only they are re-ranked by exact FP32
 * distance.  When C <= exact_rerank every candidate survives and the result
 * equals FP32's. */
#define SUCO_PRECISION_FP32 0
#define SUCO_PRECISION_BF16 1
/* FP8 (not in the paper): the same coarse pass from the index's FP8 E4M3 copy,
 * each value stored as e4m3(x / s_i) with one FP32 scale s_i = max|x| / 448
 * per subspace i (quotient in FP32, round to nearest even, saturating), and
 * decoded as code * s_i in FP32. */
#define SUCO_PRECISION_FP8 2

/* suco_query_params.rank_precision: how the half-subspace centroid distances
 * that rank the IMI cells (Algorithm 4, then Algorithm 3) are computed.
 * FP32: sum of squared differences on CUDA cores, in dimension order.
 * BF16 (not in the paper): query and centroids rounded to BF16, the inner
 * products on the tensor cores (tcgen05, FP32 accumulation), the distance
 * |q|^2 - 2<q,c> + |c|^2 with the norms of the rounded vectors summed in FP32.
 * It runs as one extra launch per RANK_CHUNK (4096) queries that writes the
 * tables into the index's workspace; calls that use it must not overlap on
 * the GPU (they share the workspace). */
#define SUCO_RANK_FP32 0
#define SUCO_RANK_BF16 1
/* FP8 (not in the paper): the same tensor-core computation with E4M3 operands
 * (tcgen05 kind::f8f6f4) and one scale per subspace: the centroids are coded
 * with the dataset's scale s_i of the FP8 copy, each query with its own
 * t_bi = (largest |q| over subspace i) / 448; the codes' products are summed on
 * the tensor cores, and the sum is multiplied by s_i * t_bi in FP32.  Needs
 * the workspace (SUCO_COPY_RANK_BF16) and the FP8 copy (SUCO_COPY_FP8). */
#define SUCO_RANK_FP8 2

typedef struct suco_query_params {
    int32_t k;            /* results per query (the maximum if k_per_query), 1..256   */
    int32_t cluster_size; /* CTAs cooperating on one query (1,2,4,8,16); 0 = automatic  */
    double alpha;         /* collision ratio, 0 < alpha <= 1                            */
    double beta;          /* re-rank ratio,   0 < beta  <= 1 (bound of beta_per_query)   */
    int32_t threads;      /* threads per CTA (256, 512 or 1024); 0 = automatic          */
    int32_t flags;        /* SUCO_QUERY_* bits, 0 by default                            */
    const int32_t* k_per_query;    /* (device, nullable) [nq], clamped to [1, k]        */
    const float* alpha_per_query;  /* (device, nullable) [nq], clamped to (0, 1]        */
    const float* beta_per_query;   /* (device, nullable) [nq], clamped to (0, beta]     */
    int32_t precision;    /* SUCO_PRECISION_*; BF16/FP8 need suco_add_reduced_copies   */
    int32_t exact_rerank; /* R: survivors of the coarse pass (0 = 512), up to 2^24       */
    int32_t id_passes;    /* passes over the id range (0 = automatic: the fewest whose
                             SC-score counters fit on chip; else a power of two); the
                             result does not depend on it                            */
    int32_t rank_precision; /* SUCO_RANK_*: arithmetic of the centroid distances that
                               rank the cells (BF16 needs suco_add_reduced_copies)    */
} suco_query_params;

/* Answers nq queries (Algorithm 4; Algorithm 3 for the cell walk).
 *   queries   (device) nq x d FP32 row-major (in the original dim order; a
 *             sampled index reads them through its permutation).
 *   out_ids   (device) nq x k int32: ids by ascending squared distance (ties
 *             by id); -1 where fewer than k candidates exist (only if n < k).
 *   out_dist  (device) nq x k FP32 squared Euclidean distances; +inf padding.
 * Asynchronous on `stream`; allocates nothing.  nq = 0 is a no-op.
 * Errors: SUCO_EINVAL (NULL pointer, k/alpha/beta out of range),
 * SUCO_EUNSUPPORTED (the per-query SC-score array of n bytes, split over the
 * cluster, or the candidate share does not fit in shared memory), SUCO_ECUDA,
 * SUCO_ETIMEOUT (the index's status word is set: see suco_read_status). */
SUCO_API int suco_query_batch(const suco_index* index, const float* queries, int64_t nq, const suco_query_params* params,
                     int32_t* out_ids, float* out_dist, void* stream);

/* Optional per-stage outputs of suco_query_debug (each pointer nullable). */
typedef struct suco_query_debug_out {
    int64_t* t_eff;      /* (device) [nq][Ns] ids collided per subspace (Algorithm 3)      */
    uint8_t* activated;  /* (device) [nq][Ns][K] 1 where the cell was retrieved            */
    float* dtab;         /* (device) [nq][Ns][2][sqrtK] FP32 squared centroid distances    */
    uint8_t* scores;     /* (device) [nq][n] SC-scores (Definition 4)                      */
    int32_t* cands;      /* (device) [nq][C] candidate ids in ascending id order: every id
                            scoring above the cut and the lowest-id ties at the cut       */
    uint8_t* survivors;  /* (device) [nq][n], zeroed by the caller: set to 1 for every
                            candidate that survives the BF16/FP8 coarse pass                */
    int64_t* stage_clock; /* (device) [nq][16][20]: row r is CTA r of the query's cluster
                            (rows past the cluster size are not written).  Slot 0: the
                            SM id; slots 1..16: the SM clock (clock64) of thread 0 at the
                            start of the query, after S0, after S1-S3, after cluster
                            barrier 1, at the start of S4, after the S4 scan, after the
                            SC-scores' bit planes, before and after cluster barrier 2,
                            after the candidate cut, before and after cluster barrier 3,
                            after the S6 distances, before and after cluster barrier 4,
                            after the merge (CTA 0 only); slots 18, 19: S4 cycles spent
                            listing segments and scanning them.  With several passes over
                            the id range, slots 6-12 hold the last pass. */
} suco_query_debug_out;

/* suco_query_batch plus the per-stage outputs above (same arguments). */
SUCO_API int suco_query_debug(const suco_index* index, const float* queries, int64_t nq, const suco_query_params* params,
                     int32_t* out_ids, float* out_dist, const suco_query_debug_out* debug, void* stream);

/* Adds reduced-precision copies of the index's dataset (no counterpart in the
 * paper).  mask bit 0 (SUCO_COPY_BF16): D rounded to BF16 (round to nearest,
 * ties to even), n x ceil8(d) 16-bit values, zero padded; it serves queries
 * with precision SUCO_PRECISION_BF16.  A copy that exists is kept.  Allocates
 * device memory; synchronous.  Errors: SUCO_EINVAL (NULL index, unknown bits),
 * SUCO_ENOMEM, SUCO_ECUDA. */
#define SUCO_COPY_BF16 1
/* mask bit 1 (SUCO_COPY_RANK_BF16): reserve the workspace of the tensor-core
 * ranking (BF16 and FP8), 4096 x Ns x 2 x sqrtK FP32 values. */
#define SUCO_COPY_RANK_BF16 2
/* mask bit 2 (SUCO_COPY_FP8): the FP8 E4M3 copy (n x ceil16(d) bytes, zero
 * padded) and its per-subspace scales; it serves SUCO_PRECISION_FP8. */
#define SUCO_COPY_FP8 4
SUCO_API int suco_add_reduced_copies(suco_index* index, int32_t mask, void* stream);

/* Times every launch shape (cluster size x threads per CTA) that fits, on the
 * given queries and parameters (which must leave cluster_size and threads at
 * 0), and remembers the fastest in the index: later calls with the same k and
 * candidate bound C and automatic shape use it.  Returns the chosen shape.
 * Synchronous; allocates two nq x k scratch outputs for the timing runs. */
SUCO_API int suco_autotune(suco_index* index, const float* queries, int64_t nq, const suco_query_params* params,
                           void* stream, int32_t* cluster_size, int32_t* threads);

/* ---- Learned per-query ratios (no counterpart in the paper, whose conclusion
 * names learning as future work).  A small MLP maps per-query features to
 * (log alpha, log beta); the query path then takes them as alpha_per_query and
 * beta_per_query.
 * Features (3*Ns per query, in this order): for each subspace i the smallest
 * squared distance to a first-half centroid and to a second-half centroid
 * (FP32, same arithmetic as the query's cell ranking), at index 2i and 2i+1;
 * then log(1 + size of the cell of those two nearest centroids) at 2Ns+i.
 * Network: xn = (x - mean) / std; z1 = xn W1 + b1; h = GELU(z1) (erf form);
 * y = h W2 + b2.  W1 [in_dim][hidden] and W2 [hidden][2] are BF16 (raw 16-bit
 * patterns), everything else FP32; every sum is FP32. */
typedef struct suco_mlp {
    int32_t in_dim;          /* 3*Ns for predict; 1..1024 for forward and backward  */
    int32_t hidden;          /* 1..4096                                             */
    int32_t out_dim;         /* must be 2                                           */
    int32_t reserved0;       /* must be 0                                           */
    const uint16_t* w1;      /* (device) [in_dim][hidden] BF16                      */
    const float* b1;         /* (device) [hidden]                                   */
    const uint16_t* w2;      /* (device) [hidden][2] BF16                           */
    const float* b2;         /* (device) [2]                                        */
    const float* feat_mean;  /* (device) [in_dim]                                   */
    const float* feat_std;   /* (device) [in_dim], nonzero                           */
    float out_offset[2];     /* margins added to y before use                       */
    float log_alpha_min, log_alpha_max, log_beta_min, log_beta_max;  /* clamps      */
    float fallback_alpha, fallback_beta;  /* used when an output is not finite      */
} suco_mlp;

/* Features of nq queries into feats (device, [nq][3*Ns]). */
SUCO_API int suco_query_features(const suco_index* index, const float* queries, int64_t nq, float* feats,
                                 void* stream);

/* Features, network and ratios in one launch: alpha[b] = exp(clamp(y0 + off0)),
 * beta[b] = exp(clamp(y1 + off1)) (device [nq] each), or the fallback ratios
 * when an output is not finite. */
SUCO_API int suco_mlp_predict(const suco_index* index, const suco_mlp* model, const float* queries, int64_t nq,
                              float* alpha, float* beta, void* stream);

/* Training pieces (device buffers; B samples of x [B][in_dim]):
 * forward writes z1, h ([B][hidden], nullable) and y [B][2]; backward takes
 * target [B][2], loss = mean over samples and outputs of (y - target)^2, and
 * writes dz1 [B][hidden] and dy [B][2] (workspace), the gradients dw1, db1,
 * dw2, db2 (FP32, same shapes as the weights; sums over samples are taken in
 * sample order) and *loss.  AdamW updates FP32 master values in place (step
 * counts from 1) and, if bf16_copy is given, writes their BF16 rounding.
 * Errors: SUCO_EINVAL for a NULL buffer, B < 1 (backward) or model sizes out
 * of range; the loss buffer is cleared by backward itself. */
SUCO_API int suco_mlp_forward(const suco_mlp* model, const float* x, int64_t B, float* z1, float* h, float* y,
                              void* stream);
SUCO_API int suco_mlp_backward(const suco_mlp* model, const float* x, int64_t B, const float* z1, const float* h,
                               const float* y, const float* target, float* dz1, float* dy, float* dw1, float* db1,
                               float* dw2, float* db2, float* loss, void* stream);
SUCO_API int suco_adamw_step(float* param, const float* grad, float* m, float* v, int64_t count, float lr,
                             float beta1, float beta2, float eps, float weight_decay, int32_t step, uint16_t* bf16_copy,
                             void* stream);

/* ---- SC-Linear (Section 3.2, Algorithm 1): the subspace-collision method
 * without the IMI.  For every query and subspace i, the T = ceil(alpha*n)
 * points nearest to q in subspace i collide, ordered by (squared subspace
 * distance, id) with the distance taken in FP32 as acc = fma(x_j - q_j,
 * x_j - q_j, acc) over the subspace's dims in order; SC-scores (Definition 4);
 * the C = ceil(beta*n) (at least k) highest scores, ties by lower id, are
 * re-ranked by exact squared distance and the k nearest returned (ties by id).
 * It reads the index's copy of D and its subspace layout (Ns), not its IMI.
 *
 * suco_sc_linear_workspace_size: bytes of device workspace that a batch of
 * `batch` queries needs (about Ns*n*4 + n bytes per query, plus 12 bytes per
 * candidate).  Host only. */
SUCO_API int suco_sc_linear_workspace_size(const suco_index* index, int64_t batch, int32_t k, double beta,
                                           size_t* bytes);

/* Answers nq queries by SC-Linear.
 *   queries    (device) nq x d FP32.   k in [1, 256].   alpha, beta in (0, 1].
 *   workspace  (device) workspace_bytes of caller-owned scratch; the call
 *              answers the queries in batches of the largest size whose
 *              workspace fits (at least one query must fit: SUCO_EINVAL
 *              otherwise).  Calls that share a workspace must not overlap.
 *   out_ids, out_dist  (device) nq x k, as suco_query_batch.
 *   dbg_scores (device, nullable) [nq][n] SC-scores; dbg_cands (device,
 *              nullable) [nq][C] candidate ids (the ids above the cut score
 *              first, in id order, then the ties at the cut in id order).
 * Asynchronous on `stream`; allocates nothing.
 * Errors: SUCO_EINVAL, SUCO_EUNSUPPORTED (Ns >= 64, a subspace longer than
 * 1600 dims, or d above 51200), SUCO_ECUDA. */
SUCO_API int suco_sc_linear(const suco_index* index, const float* queries, int64_t nq, int32_t k, double alpha,
                            double beta, void* workspace, size_t workspace_bytes, int32_t* out_ids, float* out_dist,
                            uint8_t* dbg_scores, int32_t* dbg_cands, void* stream);

/* Sizes of an index. */
typedef struct suco_index_info {
    int64_t n;
    int32_t d;
    int32_t Ns;
    int32_t sqrtK;
    int32_t hmax;      /* centroid row length in the exported layout            */
    int64_t K;         /* sqrtK^2 cells per subspace                            */
    int64_t ld;        /* row stride of the index's copy of D, in floats        */
    int64_t device_bytes;
    int32_t metric;    /* SUCO_METRIC_*                                         */
    int32_t sampled;   /* 1 when the subspaces follow a dim_perm                */
} suco_index_info;

SUCO_API int suco_index_get_info(const suco_index* index, suco_index_info* info);

/* Copies the index to host buffers (each nullable):
 *   centroids [Ns][2][sqrtK][hmax] FP32;  cell_off [Ns][K+1] uint32 offsets
 *   into perm;  perm [Ns][n] int32 ids grouped by cell.  Synchronous. */
SUCO_API int suco_export_index(const suco_index* index, float* centroids, uint32_t* cell_off, int32_t* perm);

/* The integer thresholds T and C that a query with (alpha, beta, k) uses on
 * an index of n points (host only). */
SUCO_API int suco_thresholds(int64_t n, double alpha, double beta, int32_t k, int64_t* T, int64_t* C);

/* K-means (Lloyd's algorithm) on one column range of a dataset, allocating
 * nothing.  The paper has no counterpart: this is the same computation that
 * suco_build_index runs for each half-subspace, offered to callers that cannot
 * allocate device memory at the time they call it -- for example a process
 * whose device memory is already handed out to its own allocator, or a caller
 * under a latency budget that rules out cudaMalloc and the device
 * synchronisation it implies.
 *   data       (device) n x d FP32 row-major; columns [dim_off, dim_off+dim_len)
 *              are clustered.
 *   k          centroids, 1 <= k <= min(n, 256); dim_len <= 128.  Larger sizes
 *              are rejected with SUCO_EUNSUPPORTED.
 *   iters      Lloyd iterations (assignment, then member means; an empty
 *              cluster keeps its centroid; ties go to the lowest index).
 *   centroids  (device) k x dim_len FP32: the initial centroids on entry, the
 *              final ones on return.
 *   assign     (device) n int32: each point's nearest final centroid.
 * The working sums and counts live in one fixed array of about 260 KB in
 * device global memory, defined in the library and held by every GPU that
 * loads it until the process exits.  All calls share that array: calls whose
 * GPU work overlaps in time (other streams, other host threads) race on it.
 * The first call on a device looks up the array's device address once.
 * Every call synchronises `stream` once (it reads the data's largest
 * magnitude back to the host to choose the fixed-point scale of the sums), so
 * no call can be captured into a CUDA graph.  The call raises, and never
 * lowers, the dynamic shared-memory limits of the K-means kernels it shares
 * with suco_build_index. */
SUCO_API int suco_kmeans_noalloc(const float* data, int64_t n, int32_t d, int32_t dim_off, int32_t dim_len,
                                 int32_t k, int32_t iters, float* centroids, int32_t* assign, void* stream);

/* Reads and clears the index's status word.  Kernels never spin without a
 * limit: a wait on the tensor-core ranking's MMA completion gives up after
 * about one second, stores SUCO_STATUS_WAIT_TIMEOUT in the word (which lives
 * in mapped host memory), and the launch ends with unreliable tables instead
 * of hanging.  While the word is set, suco_query_batch and suco_query_debug on
 * that index return SUCO_ETIMEOUT without launching (a wait that gives up
 * inside a call's own launch is seen by the next call, or by the same call
 * when the word was set before its query launch).  0 means every launch since
 * the last read completed normally.  Synchronises the device. */
#define SUCO_STATUS_WAIT_TIMEOUT 1u
SUCO_API int suco_read_status(suco_index* index, uint32_t* status);

/* Failure injection for tests (no counterpart in the paper).  Arms one fault,
 * process-wide, that fires at the `after`-th event of its kind from now (0 =
 * the next one) and then disarms itself:
 *   SUCO_FAULT_ALLOC         an allocation (device memory, the pinned status
 *                            word, or the host index object) fails as an
 *                            out-of-memory would: the call returns SUCO_ENOMEM
 *                            and releases what it had allocated;
 *   SUCO_FAULT_LAUNCH        a kernel launch reports failure (the query kernel
 *                            is then not launched): SUCO_ECUDA;
 *   SUCO_FAULT_WAIT_TIMEOUT  the tensor-core ranking launch behaves as if its
 *                            bounded wait had given up: it writes no tables and
 *                            sets the index's status word, which the query
 *                            entry point reports as SUCO_ETIMEOUT.
 * SUCO_FAULT_NONE disarms.  Nothing here faults, traps or stalls a GPU.
 * Errors: SUCO_EINVAL for an unknown kind or after < 0. */
#define SUCO_FAULT_NONE 0
#define SUCO_FAULT_ALLOC 1
#define SUCO_FAULT_LAUNCH 2
#define SUCO_FAULT_WAIT_TIMEOUT 3
SUCO_API int suco_inject_fault(int32_t kind, int32_t after);

/* Releases the index and its device memory.  NULL-safe. */
SUCO_API void suco_free(suco_index* index);

/* Message of the calling thread's last failed call ("" if none). */
SUCO_API const char* suco_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
SUCO_API int suco_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SUCO_H */
