"""Parity at the benchmark's full size: 1,000,000 SIFT-like points (d=128),
Ns=8, sqrtK=50, alpha=0.05, beta=0.005, k=50, one batch of 1024 queries in the
launch configuration the benchmark times.

The oracle builds its own index (one Lloyd iteration: the query path's parity
does not depend on how well K-means converged) and the GPU loads it.  Sampled
queries are compared stage by stage; every query of the batch is checked
against properties that hold at any size.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2411_14754_gb300 as pkg
from paper_2411_14754_gb300 import workloads as W
from parity_util import check_query_against_oracle, true_sqdist

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    from paper_2411_14754_gb300 import build
    build.build()
    w = W.WORKLOADS[2]
    X = W.dataset(2)
    Q = W.queries(2, nq=w.batch)
    idx = oracle.build_index(X, w.Ns, w.sqrtK, 1, W.kmeans_init_ids(2, w.n, w.Ns, w.sqrtK))
    dev = torch.device("cuda")
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).to(dev), w.Ns, w.sqrtK, idx["centroids"],
                                               idx["assign"])
    yield w, X, Q, idx, ix
    pkg.suco_free(ix)


def test_full_batch_sampled_stage_parity(full):
    w, X, Q, idx, ix = full
    dev = torch.device("cuda")
    Qd = torch.from_numpy(Q).to(dev)
    ids, dist = pkg.suco_query_batch(ix, Qd, w.k, w.alpha, w.beta)       # the benchmark's launch
    torch.cuda.synchronize()
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
    sample = [0, 137, 401, 666, 1023]
    dbg = pkg.suco_query_debug(ix, Qd[sample], w.k, w.alpha, w.beta)
    torch.cuda.synchronize()
    host = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in dbg.items()}
    T, C = host["T"], host["C"]
    assert (T, C) == (50_000, 5_000)
    for j, b in enumerate(sample):
        o = check_query_against_oracle(X, idx, Q[b], host, j, w.k, T, C)
        # the batched launch returns the same answer as the sampled launch
        assert ids[b].tolist() == host["ids"][j].tolist()
        np.testing.assert_array_equal(dist[b], host["dist"][j])
        assert o["teff"].min() >= T


def test_full_batch_properties(full):
    w, X, Q, idx, ix = full
    dev = torch.device("cuda")
    ids, dist = pkg.suco_query_batch(ix, torch.from_numpy(Q).to(dev), w.k, w.alpha, w.beta)
    torch.cuda.synchronize()
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
    assert (ids >= 0).all() and (ids < w.n).all()
    for b in range(len(Q)):
        assert len(set(ids[b].tolist())) == w.k
        assert (np.diff(dist[b]) >= 0).all()
    # integer data: every FP32 squared distance is exact
    rows = np.arange(0, len(Q), 7)
    for b in rows:
        np.testing.assert_array_equal(dist[b].astype(np.float64), true_sqdist(X, Q[b], ids[b]))


@pytest.fixture(scope="module")
def large():
    """4,000,000 points, d=16: the SC-score counters of one query (4 bits per
    id) no longer fit one pass of a 16-CTA cluster at two CTAs per SM, so the
    automatic launch takes several passes over the id range."""
    from paper_2411_14754_gb300 import build
    build.build()
    n, d, Ns, sk = 4_000_000, 16, 4, 20
    rng = np.random.default_rng(77)
    centres = rng.uniform(0, 100, size=(500, d))
    X = (centres[rng.integers(0, 500, size=n)] + rng.normal(0, 3.0, size=(n, d))).astype(np.float32)
    Q = (centres[rng.integers(0, 500, size=256)] + rng.normal(0, 3.0, size=(256, d))).astype(np.float32)
    idx = oracle.build_index(X, Ns, sk, 1, W.random_init_ids(78, n, Ns, sk))
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).cuda(), Ns, sk, idx["centroids"], idx["assign"])
    yield X, Q, idx, ix
    pkg.suco_free(ix)


def test_large_index_in_several_passes_sampled_stage_parity(large):
    X, Q, idx, ix = large
    k, alpha, beta = 10, 0.02, 0.002
    Qd = torch.from_numpy(Q).cuda()
    ids, dist = pkg.suco_query_batch(ix, Qd, k, alpha, beta)
    torch.cuda.synchronize()
    sample = [0, 77, 255]
    dbg = pkg.suco_query_debug(ix, Qd[sample], k, alpha, beta, want=("t_eff", "scores", "cands"))
    torch.cuda.synchronize()
    host = {kk: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for kk, v in dbg.items()}
    for j, b in enumerate(sample):
        check_query_against_oracle(X, idx, Q[b], host, j, k, host["T"], host["C"])
        assert ids[b].cpu().tolist() == host["ids"][j].tolist()
    # the same answer from an explicit single pass on 1024-thread CTAs
    one = pkg.suco_query_batch(ix, Qd, k, alpha, beta, id_passes=1, threads=1024, cluster_size=16)
    torch.cuda.synchronize()
    assert torch.equal(one[0], ids) and torch.equal(one[1], dist)
