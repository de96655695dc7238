"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these tests touches the CUDA library.  Each pin is chosen so that a
plausible slip in the oracle (a dropped term, a wrong index, a flipped sort
order, an off-by-one threshold) fails at least one of them.
"""
import heapq
import json
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
from paper_2411_14754_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def exact_knn(X, q, k):
    """Textbook brute force through scipy (a library routine), ties by id."""
    d = cdist(q[None, :].astype(np.float64), X.astype(np.float64), "sqeuclidean")[0]
    order = np.lexsort((np.arange(len(d)), d))[:k]
    return order, d[order]


# ---------------------------------------------------------------------------
# Definition 3 layout and the threshold reading

def test_subspace_layout_remainder_goes_last():
    # Definition 3: floor(d/Ns) dims per subspace, the last one takes the rest
    assert [oracle.subspace_dims(10, 3, i) for i in range(3)] == [(0, 3), (3, 3), (6, 4)]
    # Algorithm 2 halves: first floor(len/2), second the rest
    assert oracle.half_dims(10, 3, 2, 0) == (6, 2) and oracle.half_dims(10, 3, 2, 1) == (8, 2)
    assert oracle.half_dims(11, 3, 2, 0) == (6, 2) and oracle.half_dims(11, 3, 2, 1) == (8, 3)
    assert oracle.hmax(11, 3) == 3 and oracle.hmax(128, 8) == 8 and oracle.hmax(960, 16) == 30


def test_thresholds():
    assert oracle.collision_threshold(0.05, 10_000) == 500
    assert oracle.collision_threshold(0.07, 100) == 7          # 0.07*100 = 7.000000000000001 in binary
    assert oracle.collision_threshold(0.0501, 10_000) == 501   # ceil of a non-integral alpha*n
    assert oracle.collision_threshold(1.0, 123) == 123
    assert oracle.collision_threshold(1e-9, 123) == 1
    assert oracle.candidate_count(0.005, 1_000_000, 50) == 5000
    assert oracle.candidate_count(0.0001, 1000, 10) == 10       # raised to k
    assert oracle.candidate_count(1.0, 100, 10) == 100
    assert oracle.candidate_count(0.5, 5, 10) == 5              # clamped to n


# ---------------------------------------------------------------------------
# Algorithm 3

def test_dynamic_activation_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "da_worked_example.json")))
    d1, d2 = np.array(g["dists1_sorted"]), np.array(g["dists2_sorted"])
    sk = len(d1)
    cells, got, rows = oracle.dynamic_activation(3, d1, d2, np.ones(sk * sk, np.int64), trace=True)
    rc = [[int(c) // sk, int(c) % sk] for c in cells]
    assert rc == g["expected_first_cells_rowcol"]
    sums = [d1[r] + d2[c] for r, c in rc]
    np.testing.assert_allclose(sums, g["expected_first_sums"], rtol=0, atol=1e-12)
    assert rows.tolist() == g["expected_active_rows_after_round"]
    assert got == 3


def _key_order(d1, d2, precision):
    """All cells sorted by (cell sum, rank in d1 order, rank in d2 order)."""
    sk = len(d1)
    r1 = np.empty(sk, int)
    r1[np.lexsort((np.arange(sk), d1))] = np.arange(sk)
    r2 = np.empty(sk, int)
    r2[np.lexsort((np.arange(sk), d2))] = np.arange(sk)
    keys = []
    for a in range(sk):
        for c in range(sk):
            s = float(np.float32(d1[a]) + np.float32(d2[c])) if precision == 1 else d1[a] + d2[c]
            keys.append((s, r1[a], r2[c], a * sk + c))
    keys.sort()
    return [k[3] for k in keys]


def _multi_sequence(d1, d2, sizes, T):
    """The IMI paper's priority-queue traversal (the baseline Algorithm 3 replaces)."""
    sk = len(d1)
    i1 = np.lexsort((np.arange(sk), d1))
    i2 = np.lexsort((np.arange(sk), d2))
    seen = set()
    heap = [(d1[i1[0]] + d2[i2[0]], 0, 0)]
    out, got = [], 0
    while heap:
        s, i, j = heapq.heappop(heap)
        seen.add((i, j))
        cell = i1[i] * sk + i2[j]
        out.append(cell)
        got += sizes[cell]
        if got >= T:
            break
        if i + 1 < sk and (j == 0 or (i + 1, j - 1) in seen):
            heapq.heappush(heap, (d1[i1[i + 1]] + d2[i2[j]], i + 1, j))
        if j + 1 < sk and (i == 0 or (i - 1, j + 1) in seen):
            heapq.heappush(heap, (d1[i1[i]] + d2[i2[j + 1]], i, j + 1))
    return out, got


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("precision", [0, 1])
def test_dynamic_activation_is_a_sorted_prefix(seed, precision):
    rng = np.random.default_rng(seed)
    sk = int(rng.integers(1, 20))
    # quantised values force many equal sums; zero-size cells are allowed
    d1 = rng.integers(0, 6, size=sk).astype(np.float64) * 0.25
    d2 = rng.integers(0, 6, size=sk).astype(np.float64) * 0.25
    sizes = rng.integers(0, 4, size=sk * sk).astype(np.int64)
    total = int(sizes.sum())
    if total == 0:
        sizes[0] = 1
        total = 1
    T = int(rng.integers(1, total + 1))
    cells, got = oracle.dynamic_activation(T, d1, d2, sizes, precision=precision)
    order = _key_order(d1, d2, precision)
    # the retrieved cells are exactly the shortest prefix of the key order reaching T
    csum = np.cumsum(sizes[order])
    m = int(np.searchsorted(csum, T) + 1)
    assert cells.tolist() == order[:m]
    assert got == int(csum[m - 1]) and got >= T and got - sizes[order[m - 1]] < T


@pytest.mark.parametrize("seed", range(8))
def test_dynamic_activation_equals_multi_sequence(seed):
    # Section 4.2: Dynamic Activation returns the same cells as Multi-sequence
    rng = np.random.default_rng(100 + seed)
    sk = int(rng.integers(2, 30))
    d1 = rng.random(sk)
    d2 = rng.random(sk)
    sizes = rng.integers(0, 50, size=sk * sk).astype(np.int64)
    T = int(rng.integers(1, int(sizes.sum()) + 1))
    cells, got = oracle.dynamic_activation(T, d1, d2, sizes)
    ms, got2 = _multi_sequence(d1, d2, sizes, T)
    assert cells.tolist() == [int(c) for c in ms] and got == got2


def test_dynamic_activation_exhausts_rows():
    # reading R2: once row 0's last column is retrieved the walk moves to row 1
    # instead of retrieving the same cell again
    cells, got = oracle.dynamic_activation(4, [0.0, 100.0, 200.0], [0.3, 0.1, 0.2], np.ones(9, np.int64))
    assert cells.tolist() == [1, 2, 0, 4] and got == 4


# ---------------------------------------------------------------------------
# Algorithm 2 (K-means and the IMI)

def test_kmeans_single_step_closed_form():
    # three tight blobs, one initial point in each: one Lloyd step lands on the blob means
    rng = np.random.default_rng(7)
    centres = np.array([[0.0, 0.0], [10.0, 0.0], [0.0, 10.0]])
    lab = rng.integers(0, 3, size=300)
    X = (centres[lab] + rng.normal(0, 0.1, size=(300, 2))).astype(np.float32)
    init = [int(np.where(lab == c)[0][0]) for c in range(3)]
    cent, assign = oracle.kmeans(X, 0, 2, 3, 1, init)
    assert (assign == lab).all()
    for c in range(3):
        np.testing.assert_allclose(cent[c], X[lab == c].astype(np.float64).mean(axis=0), rtol=0, atol=1e-12)


def test_kmeans_assignment_is_argmin_and_objective_decreases():
    X = W.dataset(1, n=2000)
    init = W.random_init_ids(3, 2000, 1, 8)[0, 0]
    prev = np.inf
    for it in range(1, 6):
        cent, assign = oracle.kmeans(X, 8, 8, 8, it, init)
        # assignment of the last step is the argmin against the previous centroids
        cprev, _ = oracle.kmeans(X, 8, 8, 8, it - 1, init)
        dd = cdist(X[:, 8:16].astype(np.float64), cprev, "sqeuclidean")
        assert (assign == np.argmin(dd, axis=1)).all()
        obj = dd[np.arange(len(X)), assign].sum()
        assert obj <= prev + 1e-6
        prev = obj


def test_kmeans_empty_cluster_keeps_centroid():
    X = np.array([[0.0], [0.0], [5.0], [5.0]], np.float32)
    # ids 0 and 1 are the same point: the second centroid never wins a point
    cent, assign = oracle.kmeans(X, 0, 1, 3, 2, [0, 1, 2])
    assert assign.tolist() == [0, 0, 2, 2]
    np.testing.assert_array_equal(cent[:, 0], [0.0, 0.0, 5.0])


def test_imi_is_a_grouping_by_cell():
    rng = np.random.default_rng(5)
    sk, n = 7, 1000
    a1 = rng.integers(0, sk, n).astype(np.int32)
    a2 = rng.integers(0, sk, n).astype(np.int32)
    off, perm = oracle.imi_from_assign(a1, a2, sk)
    assert sorted(perm.tolist()) == list(range(n))
    for c in range(sk * sk):
        seg = perm[off[c]:off[c + 1]]
        assert (np.diff(seg) > 0).all()
        assert ((a1[seg] * sk + a2[seg]) == c).all()
    assert off[-1] == n


def test_build_index_final_assignment_matches_stored_centroids():
    X = W.dataset(1, n=3000)
    Ns, sk = 4, 6
    init = W.random_init_ids(11, 3000, Ns, sk)
    idx = oracle.build_index(X, Ns, sk, 3, init)
    for i in range(Ns):
        for h in range(2):
            off, ln = oracle.half_dims(128, Ns, i, h)
            c = idx["centroids"][i, h, :, :ln].astype(np.float64)
            dd = cdist(X[:, off:off + ln].astype(np.float64), c, "sqeuclidean")
            assert (idx["assign"][i, h] == np.argmin(dd, axis=1)).all()
            cent, _ = oracle.kmeans(X, off, ln, sk, 3, init[i, h])
            np.testing.assert_array_equal(idx["centroids"][i, h, :, :ln], cent.astype(np.float32))


# ---------------------------------------------------------------------------
# Algorithm 4 against independent references

def _small_index(X, Ns, sk, iters=5, seed=1):
    return oracle.build_index(X, Ns, sk, iters, W.random_init_ids(seed, X.shape[0], Ns, sk))


def test_bruteforce_matches_scipy():
    X = W.dataset(1, n=1500)
    q = W.queries(1, nq=3)
    for qq in q:
        ids, dist = oracle.bruteforce_knn(X, qq, 20)
        ref_ids, ref_d = exact_knn(X, qq, 20)
        assert ids.tolist() == ref_ids.tolist()
        np.testing.assert_allclose(dist, ref_d, rtol=1e-12)


@pytest.mark.parametrize("prec", [0, 1])
def test_alpha_one_gives_every_point_score_Ns(prec):
    X = W.dataset(1, n=1200)
    idx = _small_index(X, 8, 5)
    q = W.queries(1, nq=1)[0]
    out = oracle.query(X, idx, q, 10, T=1200, C_=50, rank_precision=prec)
    assert (out["scores"] == 8).all()
    assert (out["teff"] == 1200).all()


@pytest.mark.parametrize("prec", [0, 1])
def test_alpha_beta_one_is_exact_knn(prec):
    X = W.dataset(1, n=900)
    idx = _small_index(X, 4, 4)
    for qq in W.queries(1, nq=4):
        out = oracle.query(X, idx, qq, 15, T=900, C_=900, rank_precision=prec)
        ref_ids, ref_d = exact_knn(X, qq, 15)
        assert out["ids"].tolist() == ref_ids.tolist()
        np.testing.assert_allclose(out["dist"], ref_d, rtol=1e-12)
        assert oracle.recall(out["ids"], ref_ids) == 1.0


def test_suco_equals_sc_linear_on_a_product_grid():
    # When every IMI cell holds exactly one point that sits on its product centroid,
    # the cell value d1+d2 is that point's exact subspace distance, so Algorithm 4
    # must reproduce Algorithm 1 (SC-Linear) exactly.
    rng = np.random.default_rng(21)
    Ns, sk, hl = 3, 9, 2
    d = Ns * 2 * hl
    n = sk * sk
    cents = rng.random((Ns, 2, sk, hl)).astype(np.float32)
    X = np.empty((n, d), np.float32)
    assign = np.empty((Ns, 2, n), np.int32)
    # point p sits in cell (p // sk, p % sk) of subspace 0, shuffled cells elsewhere
    for i in range(Ns):
        cell_of = rng.permutation(n)
        for p in range(n):
            a1, a2 = divmod(int(cell_of[p]), sk)
            X[p, i * 2 * hl:i * 2 * hl + hl] = cents[i, 0, a1]
            X[p, i * 2 * hl + hl:(i + 1) * 2 * hl] = cents[i, 1, a2]
            assign[i, 0, p], assign[i, 1, p] = a1, a2
    idx = oracle.index_from_parts(Ns, sk, cents, assign)
    for T in (1, 5, 17, 40):
        q = rng.random(d).astype(np.float32)
        a = oracle.query(X, idx, q, 5, T=T, C_=10, rank_precision=0)
        ids, dist, sc = oracle.sc_linear(X, Ns, q, 5, T, 10)
        assert (a["scores"] == sc).all()
        assert (a["teff"] == T).all()
        assert a["ids"].tolist() == ids.tolist()


def test_score_invariants_and_collision_counts():
    X = W.dataset(1, n=3000)
    idx = _small_index(X, 8, 6)
    K = 36
    maxcell = max(int(np.diff(idx["cell_off"][i]).max()) for i in range(8))
    for qq in W.queries(1, nq=3):
        T = oracle.collision_threshold(0.05, 3000)
        out = oracle.query(X, idx, qq, 10, T=T, C_=50)
        s = out["scores"]
        assert s.min() >= 0 and s.max() <= 8                         # Definition 4
        assert s.sum() == out["teff"].sum()                            # every collision counted once
        assert (out["teff"] >= T).all() and (out["teff"] < T + maxcell).all()
        for i in range(8):                                             # teff = size of the retrieved cells
            sizes = np.diff(idx["cell_off"][i])
            assert out["teff"][i] == sizes[out["activated"][i].astype(bool)].sum()
        # score of a point = number of subspaces whose retrieved cells contain it
        cellid = idx["assign"][:, 0, :] * 6 + idx["assign"][:, 1, :]
        hit = np.stack([out["activated"][i][cellid[i]] for i in range(8)])
        assert (hit.sum(axis=0) == s).all()
        assert out["activated"].shape == (8, K)


def test_monotone_in_alpha_and_nested_in_beta():
    X = W.dataset(1, n=2500)
    idx = _small_index(X, 8, 6)
    q = W.queries(1, nq=1)[0]
    prev = None
    for a in (0.01, 0.03, 0.05, 0.2, 0.6):
        out = oracle.query(X, idx, q, 10, T=oracle.collision_threshold(a, 2500), C_=40)
        if prev is not None:
            assert (out["scores"] >= prev).all()
        prev = out["scores"]
    base = oracle.query(X, idx, q, 10, T=125, C_=100)["cands"]
    for c in (10, 40, 70):
        assert oracle.query(X, idx, q, 10, T=125, C_=c)["cands"].tolist() == base[:c].tolist()


def test_candidates_and_rerank_against_brute_force():
    X = W.dataset(1, n=2000)
    idx = _small_index(X, 8, 5)
    q = W.queries(1, nq=1)[0]
    out = oracle.query(X, idx, q, 12, T=100, C_=60)
    s = out["scores"]
    ref = np.lexsort((np.arange(len(s)), -s))[:60]
    assert out["cands"].tolist() == ref.tolist()
    sub = X[out["cands"]]
    rid, rd = exact_knn(sub, q, 12)
    assert out["ids"].tolist() == out["cands"][rid].tolist()
    np.testing.assert_allclose(out["dist"], rd, rtol=1e-12)


def test_select_candidates_ties_by_id():
    s = np.array([2, 3, 3, 1, 3, 2, 0], np.int32)
    assert oracle.select_candidates(s, 4).tolist() == [1, 2, 4, 0]
    assert oracle.select_candidates(s, 7).tolist() == [1, 2, 4, 0, 5, 3, 6]


def test_padding_when_fewer_candidates_than_k():
    X = W.random_data(3, 5, 6)
    ids, dist = oracle.rerank(X, X[0], np.arange(5), 8)
    assert ids[5:].tolist() == [-1, -1, -1] and np.isinf(dist[5:]).all() and ids[0] == 0


def test_fp32_ranking_equals_fp64_on_exact_data():
    # small integers with integer centroids: every FP32 operation is exact, so the
    # kernel-precision ranking and the FP64 ranking must take identical decisions
    X = W.random_data(9, 3000, 16, kind="int")
    idx = oracle.build_index(X, 4, 6, 0, W.random_init_ids(9, 3000, 4, 6))
    for qq in W.random_data(10, 5, 16, kind="int"):
        a = oracle.query(X, idx, qq, 10, T=150, C_=30, rank_precision=0)
        b = oracle.query(X, idx, qq, 10, T=150, C_=30, rank_precision=1)
        for key in ("scores", "cands", "teff", "activated", "ids"):
            assert (a[key] == b[key]).all(), key


def test_fp32_ranking_rounds_like_the_kernel():
    # two cells whose FP64 sums differ by less than half an FP32 ulp of 1.0 tie in FP32;
    # the tie then goes to the lower d1 rank (reading R3 / key order)
    d1 = np.array([1.0, 1.0 + 2.0 ** -20])
    d2 = np.array([2.0 ** -22, 0.75])
    sizes = np.ones(4, np.int64)
    c64, _ = oracle.dynamic_activation(2, d1, d2, sizes, precision=0)
    c32, _ = oracle.dynamic_activation(2, d1, d2, sizes, precision=1)
    assert c64.tolist() == [0, 2] and c32.tolist() == [0, 2]
    d2b = np.array([2.0 ** -25, 0.75])   # 1 + 2^-25 rounds to 1.0 in FP32
    d1b = np.array([1.0 + 2.0 ** -26, 1.0])
    c64, _ = oracle.dynamic_activation(1, d1b, d2b, sizes, precision=0)
    c32, _ = oracle.dynamic_activation(1, d1b, d2b, sizes, precision=1)
    assert c64.tolist() == [2]          # (row of d1=1.0) wins exactly
    assert c32.tolist() == [2]          # both FP32 sums equal 1.0: rank order decides (d1=1.0 ranks first)


def test_recall_and_mre_definitions():
    assert oracle.recall([[1, 2, 3, 4]], [[4, 3, 9, 8]]) == 0.5
    # MRE is on Euclidean (not squared) distances: result 2 vs truth 1 and 3 vs 3
    assert abs(oracle.mre([[4.0, 9.0]], [[1.0, 9.0]]) - 0.5) < 1e-12


def test_batch_driver_matches_single_queries():
    X = W.dataset(1, n=1500)
    idx = _small_index(X, 8, 5)
    Q = W.queries(1, nq=6)
    ids, dist = oracle.query_batch(X, idx, Q, 7, T=75, C_=30, nthreads=3)
    for b in range(6):
        o = oracle.query(X, idx, Q[b], 7, T=75, C_=30, debug=False)
        assert ids[b].tolist() == o["ids"].tolist()
        np.testing.assert_array_equal(dist[b], o["dist"])
    # one (T, C) per query
    Ts, Cs = [40, 75, 120, 75, 300, 9], [30, 12, 60, 7, 90, 25]
    ids, dist = oracle.query_batch(X, idx, Q, 7, T=Ts, C_=Cs, nthreads=3)
    for b in range(6):
        o = oracle.query(X, idx, Q[b], 7, T=Ts[b], C_=Cs[b], debug=False)
        assert ids[b].tolist() == o["ids"].tolist()
        np.testing.assert_array_equal(dist[b], o["dist"])


# ---------------------------------------------------------------------------
# Algorithm 4 from given half-subspace distance tables (Algorithm 4 computes
# the tables, then ranks cells from them; the tensor-core ranking's parity
# goes through this entry)

_STAGES = ("teff", "activated", "scores", "cands", "ids", "dist")


def test_query_from_tables_given_the_queries_own_tables_equals_the_query():
    X = W.random_data(31, 2500, 24, kind="gauss")
    idx = _small_index(X, 3, 6, iters=3, seed=32)
    for qq in W.random_data(33, 6, 24, kind="gauss"):
        o = oracle.query(X, idx, qq, 9, T=200, C_=40, rank_precision=1)
        t = oracle.query_from_tables(X, idx, qq, 9, T=200, C_=40, dtab=o["dtab"])
        for key in _STAGES:
            np.testing.assert_array_equal(t[key], o[key], err_msg=key)


def test_query_from_tables_written_from_the_definition_equals_the_fp64_query():
    # integer rows and integer centroids (no Lloyd update): every half-subspace
    # squared distance is an integer below 2^24, exact in FP32 and FP64.  The
    # tables are written here from the definition (per half, sum of squared
    # differences over the half's dims); ranking from them must reproduce the
    # FP64 query in every stage, and the FP64 query's own tables must equal them.
    n, d, Ns, sk = 2000, 22, 3, 5          # d not a multiple of Ns: the last subspace is longer
    X = W.random_data(34, n, d, kind="int")
    idx = _small_index(X, Ns, sk, iters=0, seed=35)
    cent = idx["centroids"].astype(np.float64)
    for qq in W.random_data(36, 5, d, kind="int"):
        tab = np.empty((Ns, 2, sk))
        for i in range(Ns):
            s = d // Ns
            off = i * s
            ln = d - (Ns - 1) * s if i == Ns - 1 else s
            halves = ((off, ln // 2), (off + ln // 2, ln - ln // 2))
            for h, (ho, hl) in enumerate(halves):
                diff = cent[i, h, :, :hl] - qq[ho:ho + hl].astype(np.float64)[None, :]
                tab[i, h] = (diff * diff).sum(axis=1)
        o = oracle.query(X, idx, qq, 8, T=120, C_=35, rank_precision=0)
        np.testing.assert_array_equal(o["dtab"], tab)
        t = oracle.query_from_tables(X, idx, qq, 8, T=120, C_=35, dtab=tab)
        for key in _STAGES:
            np.testing.assert_array_equal(t[key], o[key], err_msg=key)
        # a transposed table (halves swapped) must change the ranking somewhere
        sw = oracle.query_from_tables(X, idx, qq, 8, T=120, C_=35, dtab=tab[:, ::-1, :].copy())
        assert not np.array_equal(sw["activated"], o["activated"])


# ---------------------------------------------------------------------------
# Algorithm 1 (SC-Linear)

def _sc_linear_brute(X, Ns, q, T, C):
    """Algorithm 1 written with library routines: per subspace the first T ids
    of a lexsort by (squared distance, id) collide; candidates are the first C
    ids by (score desc, id asc)."""
    n, d = X.shape
    s = d // Ns
    scores = np.zeros(n, np.int64)
    for i in range(Ns):
        off, ln = i * s, (d - (Ns - 1) * s if i == Ns - 1 else s)
        dist = cdist(q[None, off:off + ln].astype(np.float64), X[:, off:off + ln].astype(np.float64),
                     "sqeuclidean")[0]
        scores[np.lexsort((np.arange(n), dist))[:T]] += 1
    return scores, np.lexsort((np.arange(n), -scores))[:C]


@pytest.mark.parametrize("precision", [0, 1])
def test_sc_linear_against_brute_force(precision):
    X = W.dataset(1, n=2500)
    for qq in W.queries(1, nq=3):
        ids, dist, sc, cands = oracle.sc_linear(X, 8, qq, 10, 125, 40, precision=precision, cands=True)
        bs, bc = _sc_linear_brute(X, 8, qq, 125, 40)
        np.testing.assert_array_equal(sc, bs)
        assert sorted(cands.tolist()) == sorted(bc.tolist())
        ri, rd = oracle.rerank(X, qq, bc, 10)
        assert ids.tolist() == ri.tolist()


def test_sc_linear_fp32_equals_fp64_on_exact_data_and_handles_ties():
    # small integers: every subspace distance is an exact integer in both
    # precisions; many equal distances test the (distance, id) order
    X = W.random_data(71, 3000, 12, kind="int")
    for qq in W.random_data(72, 4, 12, kind="int"):
        a = oracle.sc_linear(X, 3, qq, 7, 300, 50, precision=0, cands=True)
        b = oracle.sc_linear(X, 3, qq, 7, 300, 50, precision=1, cands=True)
        bs, bc = _sc_linear_brute(X, 3, qq, 300, 50)
        for r in (a, b):
            np.testing.assert_array_equal(r[2], bs)
            np.testing.assert_array_equal(np.sort(r[3]), np.sort(bc))


def test_sc_linear_alpha_one_and_alpha_beta_one():
    X = W.dataset(1, n=800)
    qq = W.queries(1, nq=1)[0]
    ids, dist, sc = oracle.sc_linear(X, 4, qq, 9, 800, 30, precision=1)
    assert (sc == 4).all()
    ids, dist, sc = oracle.sc_linear(X, 4, qq, 9, 800, 800, precision=1)
    ei, ed = exact_knn(X, qq, 9)
    assert ids.tolist() == ei.tolist()


# ---------------------------------------------------------------------------
# Variants: L1 distance (Section 5, SuCo-L1) and Definition 3's random
# subspace sampling

def _sc_linear_brute_dims(X, dims, q, T, C, metric):
    """Algorithm 1 written from Definition 3's dim lists with library
    routines, in either metric."""
    n = X.shape[0]
    scores = np.zeros(n, np.int64)
    kind = "cityblock" if metric == 1 else "sqeuclidean"
    for dl in dims:
        dist = cdist(q[None, dl].astype(np.float64), X[:, dl].astype(np.float64), kind)[0]
        scores[np.lexsort((np.arange(n), dist))[:T]] += 1
    return scores, np.lexsort((np.arange(n), -scores))[:C]


def test_sampled_subspaces_follow_definition_3():
    rng = np.random.default_rng(91)
    perm = rng.permutation(23)
    dims = oracle.sampled_subspaces(perm, 4)
    assert [len(x) for x in dims] == [5, 5, 5, 8]              # floor(23/4), the last takes the rest
    assert sorted(np.concatenate(dims).tolist()) == list(range(23))
    with pytest.raises(AssertionError):
        oracle.sampled_subspaces([0, 1, 1, 3], 2)


@pytest.mark.parametrize("metric", [0, 1])
def test_sc_linear_with_sampled_subspaces_and_metric_against_brute_force(metric):
    X = W.dataset(1, n=2000)
    perm = np.random.default_rng(92).permutation(X.shape[1])
    dims = oracle.sampled_subspaces(perm, 8)
    for qq in W.queries(1, nq=3):
        ids, dist, sc, cands = oracle.sc_linear(X, 8, qq, 10, 100, 40, precision=0, cands=True, metric=metric,
                                                dim_perm=perm)
        bs, bc = _sc_linear_brute_dims(X, dims, qq, 100, 40, metric)
        np.testing.assert_array_equal(sc, bs)
        assert sorted(cands.tolist()) == sorted(bc.tolist())


def test_l1_query_alpha_beta_one_is_exact_l1_knn():
    X = W.dataset(1, n=1500)
    idx = oracle.build_index(X, 4, 4, 3, W.random_init_ids(93, 1500, 4, 4), metric=1)
    for qq in W.queries(1, nq=3):
        o = oracle.query(X, idx, qq, 10, T=1500, C_=1500, rank_precision=0)
        d = cdist(qq[None, :].astype(np.float64), X.astype(np.float64), "cityblock")[0]
        order = np.lexsort((np.arange(len(d)), d))[:10]
        assert o["ids"].tolist() == order.tolist()
        np.testing.assert_allclose(o["dist"], d[order], rtol=1e-12)
        assert (o["scores"] == 4).all()


def test_l1_kmeans_assignment_is_the_l1_argmin():
    X = W.dataset(1, n=1200)
    init = np.arange(0, 1200, 100)
    cent, assign = oracle.kmeans(X, 8, 8, len(init), 1, init, metric=1)
    # after one step: the assignment used the initial points, by L1
    d = cdist(X[:, 8:16].astype(np.float64), X[init][:, 8:16].astype(np.float64), "cityblock")
    np.testing.assert_array_equal(assign, d.argmin(axis=1))
    for a in range(len(init)):
        if (assign == a).any():
            np.testing.assert_allclose(cent[a], X[assign == a][:, 8:16].astype(np.float64).mean(0), rtol=1e-12)


@pytest.mark.parametrize("metric", [0, 1])
def test_suco_equals_sc_linear_on_a_product_grid_in_both_metrics(metric):
    # every cell holds one point on its product centroid: the cell value is the
    # point's exact subspace distance (in L1 as well: it is additive)
    rng = np.random.default_rng(94)
    Ns, sk, hl = 3, 7, 2
    d, n = Ns * 2 * hl, sk * sk
    cents = rng.random((Ns, 2, sk, hl)).astype(np.float32)
    X = np.empty((n, d), np.float32)
    assign = np.empty((Ns, 2, n), np.int32)
    for i in range(Ns):
        cells = rng.permutation(n)
        for p in range(n):
            a1, a2 = divmod(int(cells[p]), sk)
            X[p, i * 2 * hl:i * 2 * hl + hl] = cents[i, 0, a1]
            X[p, i * 2 * hl + hl:(i + 1) * 2 * hl] = cents[i, 1, a2]
            assign[i, 0, p], assign[i, 1, p] = a1, a2
    idx = oracle.index_from_parts(Ns, sk, cents, assign, metric=metric)
    for qq in rng.random((4, d)).astype(np.float32):
        a = oracle.query(X, idx, qq, 5, 12, 10, rank_precision=0)
        ids, dist, sc = oracle.sc_linear(X, Ns, qq, 5, 12, 10, metric=metric)
        assert (a["scores"] == sc).all()
        assert a["ids"].tolist() == ids.tolist()


def test_sampling_that_only_reorders_dims_inside_halves_changes_nothing_on_exact_data():
    # Definition 3 treats a subspace as a set of dims: reordering the dims of
    # each half (integer data, exact in FP64) leaves every stage unchanged
    X = W.random_data(95, 2000, 16, kind="int")
    rng = np.random.default_rng(96)
    perm = np.concatenate([rng.permutation(np.arange(h * 2, h * 2 + 2)) for h in range(8)])  # 4 subspaces, halves of 2
    init = W.random_init_ids(97, 2000, 4, 5)
    a = oracle.build_index(X, 4, 5, 0, init)
    b = oracle.build_index(X, 4, 5, 0, init, dim_perm=perm)
    for qq in W.random_data(98, 4, 16, kind="int"):
        oa = oracle.query(X, a, qq, 8, 100, 30, rank_precision=0)
        ob = oracle.query(X, b, qq, 8, 100, 30, rank_precision=0)
        for key in ("teff", "activated", "scores", "ids", "dist"):
            np.testing.assert_array_equal(oa[key], ob[key], err_msg=key)
