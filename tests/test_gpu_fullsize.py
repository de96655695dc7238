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
