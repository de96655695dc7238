"""The paper's variants on the GPU vs the CPU oracle, through the C ABI:
the L1 distance (Section 5's SuCo-L1) and Definition 3's random subspace
sampling, for the index build, the query path (every stage), SC-Linear and
the learned features.  Decisions are compared in the kernels' FP32
arithmetic (bit-exact); returned distances within 1e-5 relative of FP64.
"""
import numpy as np
import pytest
import torch
from scipy.spatial.distance import cdist

import oracle
import paper_2411_14754_gb300 as pkg
from oracle import mlp_oracle as M
from paper_2411_14754_gb300 import workloads as W
from parity_util import RTOL, assert_topk_matches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2411_14754_gb300 import build
    build.build()
    pkg.load_library()


def l1_dist(X, q, ids):
    ids = np.asarray(ids)
    out = np.full(len(ids), np.inf)
    ok = ids >= 0
    out[ok] = np.abs(X[ids[ok]].astype(np.float64) - q.astype(np.float64)[None, :]).sum(1)
    return out


def assert_topk_matches_l1(X, q, gids, gdist, oids, odist):
    gids, oids = np.asarray(gids, np.int64), np.asarray(oids, np.int64)
    assert ((gids < 0) == (oids < 0)).all()
    real = gids >= 0
    np.testing.assert_allclose(np.asarray(gdist, np.float64)[real], l1_dist(X, q, gids[real]), rtol=RTOL)
    np.testing.assert_allclose(np.asarray(gdist, np.float64)[real], np.asarray(odist)[real], rtol=RTOL)
    dk = float(np.asarray(odist)[real][-1])
    for i in set(gids[real].tolist()) ^ set(oids[real].tolist()):
        assert abs(l1_dist(X, q, [i])[0] - dk) <= 2 * RTOL * dk


def gpu_index(X, idx, metric, perm):
    return pkg.suco_build_index_from_parts(torch.from_numpy(np.ascontiguousarray(X)).cuda(), idx["Ns"], idx["sqrtK"],
                                           idx["centroids"], idx["assign"], metric=metric, dim_perm=perm)


CASES = [("l1", False), ("l2", True), ("l1", True)]


@pytest.mark.parametrize("metric,sampled", CASES)
def test_query_stages_match_the_oracle(metric, sampled):
    w = W.WORKLOADS[1]
    X = W.dataset(1)
    Q = W.queries(1, nq=60)
    perm = np.random.default_rng(101).permutation(w.d) if sampled else None
    idx = oracle.build_index(X, w.Ns, w.sqrtK, 5, W.kmeans_init_ids(1, w.n, w.Ns, w.sqrtK),
                             metric=oracle.METRIC_L1 if metric == "l1" else 0, dim_perm=perm)
    ix = gpu_index(X, idx, metric, perm)
    try:
        assert ix.metric == (1 if metric == "l1" else 0) and ix.sampled == (1 if sampled else 0)
        Qd = torch.from_numpy(Q).cuda()
        out = pkg.suco_query_debug(ix, Qd, w.k, 0.05, 0.01)
        full = pkg.suco_query_batch(ix, Qd, w.k, 0.05, 0.01)
        torch.cuda.synchronize()
        host = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in out.items()}
    finally:
        pkg.suco_free(ix)
    assert np.array_equal(full[0].cpu().numpy(), host["ids"])
    T, C = host["T"], host["C"]
    for b in range(len(Q)):
        o = oracle.query(X, idx, Q[b], w.k, T, C, rank_precision=1, debug=True)
        np.testing.assert_array_equal(host["dtab"][b].astype(np.float64), o["dtab"])
        np.testing.assert_array_equal(host["t_eff"][b], o["teff"])
        np.testing.assert_array_equal(host["activated"][b], o["activated"])
        np.testing.assert_array_equal(host["scores"][b].astype(np.int32), o["scores"])
        assert sorted(host["cands"][b].tolist()) == sorted(o["cands"].tolist())
        if metric == "l1":
            assert_topk_matches_l1(X, Q[b], host["ids"][b], host["dist"][b], o["ids"], o["dist"])
        else:
            assert_topk_matches(X, Q[b], host["ids"][b], host["dist"][b], o["ids"], o["dist"])


@pytest.mark.parametrize("metric,sampled", CASES)
def test_gpu_build_follows_the_metric_and_the_sampling(metric, sampled):
    # Lloyd's iterations on the GPU against the oracle's: the same initial
    # points, one iteration (assignment under the metric, then member means);
    # the IMI of the GPU's own centroids must be the assignment under the metric
    w = W.WORKLOADS[1]
    X = W.dataset(1)
    perm = np.random.default_rng(102).permutation(w.d) if sampled else None
    m = oracle.METRIC_L1 if metric == "l1" else 0
    init = W.kmeans_init_ids(1, w.n, w.Ns, w.sqrtK)
    ix = pkg.suco_build_index(torch.from_numpy(X).cuda(), w.Ns, w.sqrtK, 1, init_ids=init, metric=metric,
                              dim_perm=perm)
    ex = pkg.suco_export_index(ix)
    pkg.suco_free(ix)
    ref = oracle.build_index(X, w.Ns, w.sqrtK, 1, init, metric=m, dim_perm=perm)
    Xp = X if perm is None else X[:, perm]
    kind = "cityblock" if m else "sqeuclidean"
    for i in range(w.Ns):
        for h in range(2):
            off, ln = oracle.half_dims(w.d, w.Ns, i, h)
            g = ex["centroids"][i, h, :, :ln].astype(np.float64)
            np.testing.assert_allclose(g, ref["centroids"][i, h, :, :ln], rtol=1e-5, atol=1e-4)
            # the GPU's cells: every point sits in the cell of its nearest GPU centroids (ties aside)
            dd = cdist(Xp[:, off:off + ln].astype(np.float64), g, kind)
            best = dd.min(axis=1)
            cells = np.empty(w.n, np.int64)
            co, pm = ex["cell_off"][i].astype(np.int64), ex["perm"][i]
            for c in range(w.sqrtK * w.sqrtK):
                cells[pm[co[c]:co[c + 1]]] = c
            a = cells // w.sqrtK if h == 0 else cells % w.sqrtK
            np.testing.assert_allclose(dd[np.arange(w.n), a], best, rtol=1e-5)


@pytest.mark.parametrize("metric,sampled", CASES)
def test_sc_linear_matches_the_oracle(metric, sampled):
    X = W.dataset(1, n=4000)
    Q = W.queries(1, nq=16)
    perm = np.random.default_rng(103).permutation(X.shape[1]) if sampled else None
    m = oracle.METRIC_L1 if metric == "l1" else 0
    ix = pkg.suco_build_index(torch.from_numpy(X).cuda(), 8, 2, 0, seed=1, metric=metric, dim_perm=perm)
    try:
        ids, dist, sc, cd = pkg.suco_sc_linear(ix, torch.from_numpy(Q).cuda(), 10, 0.05, 0.01, debug=True)
        torch.cuda.synchronize()
        T, C = pkg.suco_thresholds(4000, 0.05, 0.01, 10)
    finally:
        pkg.suco_free(ix)
    for b in range(len(Q)):
        oi, od, osc, oc = oracle.sc_linear(X, 8, Q[b], 10, T, C, precision=1, cands=True, metric=m, dim_perm=perm)
        np.testing.assert_array_equal(sc[b].cpu().numpy().astype(np.int32), osc)
        assert sorted(cd[b].cpu().tolist()) == sorted(oc.tolist())
        if metric == "l1":
            assert_topk_matches_l1(X, Q[b], ids[b].cpu().numpy(), dist[b].cpu().numpy(), oi, od)
        else:
            assert_topk_matches(X, Q[b], ids[b].cpu().numpy(), dist[b].cpu().numpy(), oi, od)


@pytest.mark.parametrize("metric,sampled", CASES)
def test_learned_features_follow_the_metric_and_the_sampling(metric, sampled):
    w = W.WORKLOADS[1]
    X = W.dataset(1, n=5000)
    Q = W.queries(1, nq=20)
    perm = np.random.default_rng(104).permutation(w.d) if sampled else None
    idx = oracle.build_index(X, w.Ns, w.sqrtK, 3, W.kmeans_init_ids(1, 5000, w.Ns, w.sqrtK),
                             metric=oracle.METRIC_L1 if metric == "l1" else 0, dim_perm=perm)
    ix = gpu_index(X, idx, metric, perm)
    try:
        f = pkg.suco_query_features(ix, torch.from_numpy(Q).cuda()).cpu().numpy()
    finally:
        pkg.suco_free(ix)
    Ns = w.Ns
    for b in range(len(Q)):
        o = M.features(X, idx, Q[b])
        np.testing.assert_array_equal(f[b, :2 * Ns].astype(np.float64), o[:2 * Ns])   # the ranking's FP32 arithmetic
        np.testing.assert_array_equal(np.rint(np.expm1(f[b, 2 * Ns:].astype(np.float64))), np.rint(np.expm1(o[2 * Ns:])))


def test_l1_index_refuses_the_squared_distance_forms():
    w = W.WORKLOADS[1]
    X = W.dataset(1, n=3000)
    ix = pkg.suco_build_index(torch.from_numpy(X).cuda(), w.Ns, 6, 1, seed=3, metric="l1")
    try:
        pkg.suco_add_reduced_copies(ix)
        Qd = torch.from_numpy(W.queries(1, nq=4)).cuda()
        for kw in (dict(precision="bf16"), dict(rank_precision="bf16"), dict(rank_precision="fp8"), dict(threads=256)):
            with pytest.raises(pkg.SucoError) as e:
                pkg.suco_query_batch(ix, Qd, 10, 0.05, 0.01, **kw)
            assert e.value.code == -6
    finally:
        pkg.suco_free(ix)


def test_dim_perm_must_be_a_permutation():
    X = torch.from_numpy(W.dataset(1, n=500)).cuda()
    bad = np.arange(128)
    bad[5] = 6
    with pytest.raises(pkg.SucoError) as e:
        pkg.suco_build_index(X, 8, 4, 1, dim_perm=bad)
    assert e.value.code == -1
