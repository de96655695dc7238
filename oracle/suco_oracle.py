"""ctypes wrapper of the C oracle in ``suco_oracle.c`` (TEST INFRASTRUCTURE).

Every function restates a step of the paper's method on the CPU in FP64 (see
the C file's header for the readings it takes).  Arrays are NumPy; nothing
here touches a GPU or the CUDA library.
"""
import ctypes as C
import os

import numpy as np

from . import build_oracle

_lib = None

_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")


def _opt(p):
    """Optional array argument (NULL when None)."""
    return p if p is not None else None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    path = build_oracle.build()
    L = C.CDLL(path)
    i32, i64, f64 = C.c_int32, C.c_int64, C.c_double
    vp = C.c_void_p
    L.orc_subspace_dims.argtypes = [i32, i32, i32, C.POINTER(i32), C.POINTER(i32)]
    L.orc_half_dims.argtypes = [i32, i32, i32, i32, C.POINTER(i32), C.POINTER(i32)]
    L.orc_hmax.argtypes = [i32, i32]
    L.orc_hmax.restype = i32
    L.orc_collision_threshold.argtypes = [f64, i64]
    L.orc_collision_threshold.restype = i64
    L.orc_candidate_count.argtypes = [f64, i64, i32]
    L.orc_candidate_count.restype = i64
    L.orc_argsort_stable.argtypes = [_f64p, i32, _i32p]
    L.orc_dynamic_activation.argtypes = [i64, i32, _f64p, _i32p, _f64p, _i32p, _i64p, i32, _i32p,
                                         C.POINTER(i64), vp]
    L.orc_dynamic_activation.restype = i64
    L.orc_select_candidates.argtypes = [_i32p, i64, i64, _i64p]
    L.orc_rerank.argtypes = [_f32p, i32, _f32p, _i64p, i64, i32, _i64p, _f64p, i32]
    L.orc_bruteforce_knn.argtypes = [_f32p, i64, i32, _f32p, i32, _i64p, _f64p, i32]
    L.orc_kmeans.argtypes = [_f32p, i64, i32, i32, i32, i32, i32, _i64p, _f64p, _i32p, i32]
    L.orc_assign_nearest.argtypes = [_f32p, i64, i32, i32, i32, _f32p, i32, i32, _i32p, i32]
    L.orc_imi_from_assign.argtypes = [_i32p, _i32p, i64, i32, _i64p, _i64p]
    L.orc_build_index.argtypes = [_f32p, i64, i32, i32, i32, i32, _i64p, _f32p, _i32p, _i64p, _i64p, i32, i32]
    L.orc_query.argtypes = [_f32p, i64, i32, i32, i32, _f32p, _i64p, _i64p, _f32p, i32, i64, i64, i32,
                            _i64p, _f64p, vp, vp, vp, vp, vp, i32]
    L.orc_query.restype = C.c_int
    L.orc_query_from_tables.argtypes = [_f32p, i64, i32, i32, i32, _f32p, _i64p, _i64p, _f32p, i32, i64, i64, _f64p,
                                        _i64p, _f64p, vp, vp, vp, vp, i32]
    L.orc_query_from_tables.restype = C.c_int
    L.orc_query_batch.argtypes = [_f32p, i64, i32, i32, i32, _f32p, _i64p, _i64p, _f32p, i64, i32, i64, i64,
                                  i32, i32, _i64p, _f64p, i32]
    L.orc_query_batch_pq.argtypes = [_f32p, i64, i32, i32, i32, _f32p, _i64p, _i64p, _f32p, i64, i32, _i64p, _i64p,
                                     i32, i32, _i64p, _f64p, i32]
    L.orc_sc_linear.argtypes = [_f32p, i64, i32, i32, _f32p, i32, i64, i64, i32, _i64p, _f64p, vp, vp, i32]
    L.orc_max_threads.restype = C.c_int
    _lib = L
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# --------------------------------------------------------------------------
# Layout and thresholds (Definition 3; Algorithm 2; reading R4)

METRIC_L2, METRIC_L1 = 0, 1


def sampled_subspaces(dim_perm, Ns):
    """Definition 3's subspaces from a sampling given as a permutation of the
    d dims: round i < Ns-1 takes the floor(d/Ns) dims dim_perm[i*s:(i+1)*s]
    (sampled without replacement: each dim at most once), the last subspace
    every remaining dim.  Returns the list of Ns dim lists."""
    perm = np.asarray(dim_perm, dtype=np.int64)
    d = len(perm)
    assert sorted(perm.tolist()) == list(range(d)), "not a permutation of the dims"
    s = d // Ns
    return [perm[i * s:(i + 1) * s] if i < Ns - 1 else perm[(Ns - 1) * s:] for i in range(Ns)]


def _columns(X, index):
    """The dataset's columns in the index's sampling order (subspace i then
    occupies the contiguous block that Definition 3's contiguous case gives it)."""
    if index is None or index.get("dim_perm") is None:
        return _f32(X)
    if "Xp" in index and index["Xp"].shape == X.shape:
        return index["Xp"]
    return np.ascontiguousarray(np.asarray(X, dtype=np.float32)[:, index["dim_perm"]])


def _query_cols(q, index):
    if index is None or index.get("dim_perm") is None:
        return _f32(q)
    return np.ascontiguousarray(np.asarray(q, dtype=np.float32)[..., index["dim_perm"]])

def subspace_dims(d, Ns, i):
    off, ln = C.c_int32(), C.c_int32()
    lib().orc_subspace_dims(d, Ns, i, C.byref(off), C.byref(ln))
    return off.value, ln.value


def half_dims(d, Ns, i, h):
    off, ln = C.c_int32(), C.c_int32()
    lib().orc_half_dims(d, Ns, i, h, C.byref(off), C.byref(ln))
    return off.value, ln.value


def hmax(d, Ns):
    return lib().orc_hmax(d, Ns)


def collision_threshold(alpha, n):
    return int(lib().orc_collision_threshold(float(alpha), int(n)))


def candidate_count(beta, n, k):
    return int(lib().orc_candidate_count(float(beta), int(n), int(k)))


# --------------------------------------------------------------------------
# Algorithm 3 and its pieces

def argsort_stable(v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    idx = np.empty(len(v), dtype=np.int32)
    lib().orc_argsort_stable(v, len(v), idx)
    return idx


def dynamic_activation(T, dists1, dists2, cell_size, precision=0, trace=False):
    """Algorithm 3.  Returns (cells in retrieval order, retrieved id count[, rows trace])."""
    d1 = np.ascontiguousarray(dists1, dtype=np.float64)
    d2 = np.ascontiguousarray(dists2, dtype=np.float64)
    sk = len(d1)
    i1, i2 = argsort_stable(d1), argsort_stable(d2)
    cs = np.ascontiguousarray(cell_size, dtype=np.int64)
    assert cs.shape == (sk * sk,)
    cells = np.empty(sk * sk, dtype=np.int32)
    tr = np.zeros(sk * sk, dtype=np.int32) if trace else None
    got = C.c_int64()
    nc = lib().orc_dynamic_activation(int(T), sk, d1, i1, d2, i2, cs, precision, cells, C.byref(got), _ptr(tr))
    if trace:
        return cells[:nc].copy(), got.value, tr[:nc].copy()
    return cells[:nc].copy(), got.value


def select_candidates(scores, C_):
    s = np.ascontiguousarray(scores, dtype=np.int32)
    out = np.empty(C_, dtype=np.int64)
    lib().orc_select_candidates(s, len(s), int(C_), out)
    return out


def rerank(X, q, ids, k, metric=METRIC_L2):
    X = _f32(X)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    oi = np.empty(k, dtype=np.int64)
    od = np.empty(k, dtype=np.float64)
    lib().orc_rerank(X, X.shape[1], _f32(q), ids, len(ids), k, oi, od, int(metric))
    return oi, od


def bruteforce_knn(X, q, k, metric=METRIC_L2):
    X = _f32(X)
    oi = np.empty(k, dtype=np.int64)
    od = np.empty(k, dtype=np.float64)
    lib().orc_bruteforce_knn(X, X.shape[0], X.shape[1], _f32(q), k, oi, od, int(metric))
    return oi, od


# --------------------------------------------------------------------------
# Algorithm 2

def kmeans(X, off, ln, k, iters, init_ids, metric=METRIC_L2):
    """Lloyd's iterations: nearest centroid under the metric, then member means."""
    X = _f32(X)
    cent = np.empty((k, ln), dtype=np.float64)
    assign = np.empty(X.shape[0], dtype=np.int32)
    lib().orc_kmeans(X, X.shape[0], X.shape[1], off, ln, k, iters,
                     np.ascontiguousarray(init_ids, dtype=np.int64), cent, assign, int(metric))
    return cent, assign


def assign_nearest(X, off, ln, cent_f32, metric=METRIC_L2):
    X = _f32(X)
    cent = _f32(cent_f32)
    out = np.empty(X.shape[0], dtype=np.int32)
    lib().orc_assign_nearest(X, X.shape[0], X.shape[1], off, ln, cent, cent.shape[0], cent.shape[1], out,
                             int(metric))
    return out


def imi_from_assign(a1, a2, sqrtK):
    a1 = np.ascontiguousarray(a1, dtype=np.int32)
    a2 = np.ascontiguousarray(a2, dtype=np.int32)
    n = len(a1)
    off = np.empty(sqrtK * sqrtK + 1, dtype=np.int64)
    perm = np.empty(n, dtype=np.int64)
    lib().orc_imi_from_assign(a1, a2, n, sqrtK, off, perm)
    return off, perm


def build_index(X, Ns, sqrtK, iters, init_ids, nthreads=None, metric=METRIC_L2, dim_perm=None):
    """Algorithm 2.  Returns a dict with centroids [Ns,2,sqrtK,hmax] (FP32),
    assign [Ns,2,n], cell_off [Ns,K+1], perm [Ns,n].  metric: the distance of
    the nearest-centroid assignments; dim_perm: Definition 3's subspace
    sampling (see sampled_subspaces), None for contiguous subspaces.  The
    centroids of subspace i are over its dims in the sampling's order."""
    if dim_perm is not None:
        sampled_subspaces(dim_perm, Ns)
        Xp = np.ascontiguousarray(np.asarray(X, dtype=np.float32)[:, np.asarray(dim_perm, dtype=np.int64)])
        idx = build_index(Xp, Ns, sqrtK, iters, init_ids, nthreads, metric)
        idx.update(dim_perm=np.asarray(dim_perm, dtype=np.int64), Xp=Xp)
        return idx
    X = _f32(X)
    n, d = X.shape
    hm = hmax(d, Ns)
    K = sqrtK * sqrtK
    init = np.ascontiguousarray(init_ids, dtype=np.int64).reshape(Ns, 2, sqrtK)
    cent = np.zeros((Ns, 2, sqrtK, hm), dtype=np.float32)
    assign = np.empty((Ns, 2, n), dtype=np.int32)
    off = np.empty((Ns, K + 1), dtype=np.int64)
    perm = np.empty((Ns, n), dtype=np.int64)
    nt = nthreads if nthreads else max(1, min(2 * Ns, os.cpu_count() or 1))
    lib().orc_build_index(X, n, d, Ns, sqrtK, iters, init, cent, assign, off, perm, nt, int(metric))
    return dict(Ns=Ns, sqrtK=sqrtK, centroids=cent, assign=assign, cell_off=off, perm=perm, metric=int(metric))


def index_from_parts(Ns, sqrtK, centroids, assign, metric=METRIC_L2):
    """The IMI (R8) of a given set of FP32 centroids and assignments."""
    assign = np.ascontiguousarray(assign, dtype=np.int32)
    n = assign.shape[2]
    K = sqrtK * sqrtK
    off = np.empty((Ns, K + 1), dtype=np.int64)
    perm = np.empty((Ns, n), dtype=np.int64)
    for i in range(Ns):
        off[i], perm[i] = imi_from_assign(assign[i, 0], assign[i, 1], sqrtK)
    return dict(Ns=Ns, sqrtK=sqrtK, centroids=_f32(centroids), assign=assign, cell_off=off, perm=perm,
                metric=int(metric))


# --------------------------------------------------------------------------
# Algorithm 4, Algorithm 1

def query(X, index, q, k, T, C_, rank_precision=1, debug=True):
    """Algorithm 4 for one query.  rank_precision 1 takes the cell-ranking
    decisions in the GPU kernel's FP32 arithmetic, 0 in FP64.  The index's
    metric and subspace sampling apply (distances are then L1 for METRIC_L1;
    results are ids of X and their distances)."""
    X = _columns(X, index)
    q = _query_cols(q, index)
    n, d = X.shape
    Ns, sk = index["Ns"], index["sqrtK"]
    K = sk * sk
    oi = np.empty(k, dtype=np.int64)
    od = np.empty(k, dtype=np.float64)
    out = dict(ids=oi, dist=od)
    if debug:
        out.update(scores=np.empty(n, dtype=np.int32), cands=np.empty(C_, dtype=np.int64),
                   teff=np.empty(Ns, dtype=np.int64), activated=np.empty((Ns, K), dtype=np.uint8),
                   dtab=np.empty((Ns, 2, sk), dtype=np.float64))
    lib().orc_query(X, n, d, Ns, sk, index["centroids"], index["cell_off"], index["perm"], _f32(q), k, int(T),
                    int(C_), rank_precision, oi, od,
                    _ptr(out.get("scores")), _ptr(out.get("cands")), _ptr(out.get("teff")),
                    _ptr(out.get("activated")), _ptr(out.get("dtab")), int(index.get("metric", 0)))
    return out


def query_from_tables(X, index, q, k, T, C_, dtab):
    """Algorithm 4 for one query with the centroid-distance tables given
    ([Ns][2][sqrtK]); the cell ranking is then taken in FP32 like the kernel's."""
    X = _columns(X, index)
    q = _query_cols(q, index)
    n, d = X.shape
    Ns, sk = index["Ns"], index["sqrtK"]
    K = sk * sk
    oi = np.empty(k, dtype=np.int64)
    od = np.empty(k, dtype=np.float64)
    out = dict(ids=oi, dist=od, scores=np.empty(n, dtype=np.int32), cands=np.empty(C_, dtype=np.int64),
               teff=np.empty(Ns, dtype=np.int64), activated=np.empty((Ns, K), dtype=np.uint8))
    tab = np.ascontiguousarray(dtab, dtype=np.float64).reshape(Ns, 2, sk)
    lib().orc_query_from_tables(X, n, d, Ns, sk, index["centroids"], index["cell_off"], index["perm"], _f32(q), k,
                                int(T), int(C_), tab, oi, od, _ptr(out["scores"]), _ptr(out["cands"]),
                                _ptr(out["teff"]), _ptr(out["activated"]), int(index.get("metric", 0)))
    return out


def query_batch(X, index, Q, k, T, C_, rank_precision=1, nthreads=1):
    """Algorithm 4 over a batch, OpenMP over queries.  T and C_ are scalars or
    one value per query."""
    X = _columns(X, index)
    Q = _query_cols(Q, index)
    n, d = X.shape
    nq = Q.shape[0]
    oi = np.empty((nq, k), dtype=np.int64)
    od = np.empty((nq, k), dtype=np.float64)
    if np.ndim(T) or np.ndim(C_):
        Tq = np.ascontiguousarray(np.broadcast_to(np.asarray(T, dtype=np.int64), (nq,)))
        Cq = np.ascontiguousarray(np.broadcast_to(np.asarray(C_, dtype=np.int64), (nq,)))
        lib().orc_query_batch_pq(X, n, d, index["Ns"], index["sqrtK"], index["centroids"], index["cell_off"],
                                 index["perm"], Q, nq, k, Tq, Cq, rank_precision, int(nthreads), oi, od,
                                 int(index.get("metric", 0)))
        return oi, od
    lib().orc_query_batch(X, n, d, index["Ns"], index["sqrtK"], index["centroids"], index["cell_off"],
                          index["perm"], Q, nq, k, int(T), int(C_), rank_precision, int(nthreads), oi, od,
                          int(index.get("metric", 0)))
    return oi, od


def sc_linear(X, Ns, q, k, T, C_, precision=0, cands=False, metric=METRIC_L2, dim_perm=None):
    """Algorithm 1 (SC-Linear).  precision 0: FP64 subspace distances; 1: the
    kernel's FP32 arithmetic.  metric: squared L2 or L1; dim_perm: Definition
    3's sampling.  Returns (ids, dist, scores[, cands])."""
    if dim_perm is not None:
        sampled_subspaces(dim_perm, Ns)
        pm = np.asarray(dim_perm, dtype=np.int64)
        X = np.asarray(X, dtype=np.float32)[:, pm]
        q = np.asarray(q, dtype=np.float32)[pm]
    X = _f32(X)
    n, d = X.shape
    oi = np.empty(k, dtype=np.int64)
    od = np.empty(k, dtype=np.float64)
    sc = np.empty(n, dtype=np.int32)
    cd = np.empty(C_, dtype=np.int64) if cands else None
    lib().orc_sc_linear(X, n, d, Ns, _f32(q), k, int(T), int(C_), int(precision), oi, od, _ptr(sc), _ptr(cd),
                        int(metric))
    return (oi, od, sc, cd) if cands else (oi, od, sc)


def max_threads():
    return lib().orc_max_threads()


# --------------------------------------------------------------------------
# Quality measures of Section 5.1

def recall(result_ids, truth_ids):
    """|R intersect R*| / k per query, averaged."""
    r = np.atleast_2d(result_ids)
    g = np.atleast_2d(truth_ids)
    k = g.shape[1]
    return float(np.mean([len(set(a.tolist()) & set(b.tolist())) / k for a, b in zip(r, g)]))


def mre(result_sqdist, truth_sqdist):
    """Mean relative error of the (Euclidean, not squared) distances."""
    r = np.sqrt(np.atleast_2d(np.asarray(result_sqdist, dtype=np.float64)))
    g = np.sqrt(np.atleast_2d(np.asarray(truth_sqdist, dtype=np.float64)))
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = np.where(g > 0, (r - g) / g, 0.0)
    return float(np.mean(rel))
