"""SC-Linear (Algorithm 1) on the GPU vs the CPU oracle, through the C ABI.

The collisions are a discrete decision taken from floating-point subspace
distances, so the oracle takes them in the kernel's FP32 arithmetic
(precision 1): SC-scores and candidate sets must then be bit-exact, and the
top-k must match the oracle's within 1e-5 relative (FP32 vs FP64 re-rank).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2411_14754_gb300 as pkg
from paper_2411_14754_gb300 import workloads as W
from parity_util import assert_topk_matches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2411_14754_gb300 import build
    build.build()
    pkg.load_library()


def check(X, Q, Ns, k, alpha, beta, batch=32, sample=None, workspace_queries=None):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    ix = pkg.suco_build_index(Xd, Ns, 2, 0, seed=1)   # SC-Linear reads only the dataset and the layout
    try:
        Qd = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
        ws = None
        if workspace_queries:
            ws = torch.empty(pkg.suco_sc_linear_workspace_size(ix, workspace_queries, k, beta), dtype=torch.uint8,
                             device="cuda")
        ids, dist, sc, cd = pkg.suco_sc_linear(ix, Qd, k, alpha, beta, workspace=ws, batch=batch, debug=True)
        plain = pkg.suco_sc_linear(ix, Qd, k, alpha, beta, workspace=ws, batch=batch)
        torch.cuda.synchronize()
        T, C = pkg.suco_thresholds(X.shape[0], alpha, beta, k)
    finally:
        pkg.suco_free(ix)
    assert torch.equal(plain[0], ids) and torch.equal(plain[1], dist)
    ids, dist, sc, cd = ids.cpu().numpy(), dist.cpu().numpy(), sc.cpu().numpy(), cd.cpu().numpy()
    for b in (range(len(Q)) if sample is None else sample):
        oi, od, osc, oc = oracle.sc_linear(X, Ns, Q[b], k, T, C, precision=1, cands=True)
        np.testing.assert_array_equal(sc[b].astype(np.int32), osc)
        assert sorted(cd[b].tolist()) == sorted(oc.tolist())
        assert_topk_matches(X, Q[b], ids[b], dist[b], oi, od)
    return T, C


def test_tiny_workload_every_query():
    w = W.WORKLOADS[1]
    check(W.dataset(1), W.queries(1), w.Ns, w.k, w.alpha, w.beta)


@pytest.mark.parametrize("alpha,beta,k", [(0.01, 0.001, 10), (0.2, 0.02, 50), (1.0, 0.005, 7), (0.05, 1.0, 5),
                                          (1.0, 1.0, 10)])
def test_ratios_and_k(alpha, beta, k):
    check(W.dataset(1, n=3000), W.queries(1, nq=12), 8, k, alpha, beta)


def test_integer_data_with_many_distance_ties():
    # distances are small integers: the cut distance is shared by many points,
    # and the last colliding id decides; scores tie at the candidate cut too
    X = W.random_data(81, 6000, 12, kind="int")
    Q = W.random_data(82, 20, 12, kind="int")
    check(X, Q, 3, 10, 0.05, 0.01)


def test_ragged_layout_and_batches():
    # d not a multiple of Ns (the last subspace is longer), n not a multiple of
    # the tiles, a workspace that holds 3 queries: 10 queries in 4 batches
    X = W.random_data(83, 5003, 29, kind="gauss")
    Q = W.random_data(84, 10, 29, kind="gauss")
    check(X, Q, 4, 9, 0.07, 0.01, workspace_queries=3)


def test_fewer_points_than_k():
    X = W.random_data(85, 6, 8, kind="gauss")
    Q = W.random_data(86, 3, 8, kind="gauss")
    check(X, Q, 2, 10, 0.5, 0.5)


def test_sift_like_million_sampled():
    w = W.WORKLOADS[2]
    X = W.dataset(2)
    Q = W.queries(2, nq=64)
    T, C = check(X, Q, w.Ns, w.k, w.alpha, w.beta, sample=[0, 31, 63])
    assert (T, C) == (50_000, 5_000)


def test_workspace_too_small_is_refused():
    X = torch.from_numpy(W.dataset(1, n=2000)).cuda()
    ix = pkg.suco_build_index(X, 8, 2, 0, seed=1)
    try:
        ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
        with pytest.raises(pkg.SucoError) as e:
            pkg.suco_sc_linear(ix, X[:2].contiguous(), 10, 0.05, 0.005, workspace=ws)
        assert e.value.code == -1
    finally:
        pkg.suco_free(ix)
