"""suco_kmeans_noalloc: K-means on one column range with no device allocation in
the library (its scratch is a fixed array defined in the library).

Callers that cannot allocate device memory when they run the step use this
entry point; its results must equal those of the K-means inside
suco_build_index, which allocates its scratch.  This file is collected last so
that, if it fails, every other test has already run.
"""
import numpy as np
import pytest
import torch

import paper_2411_14754_gb300 as pkg
from paper_2411_14754_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2411_14754_gb300 import build
    build.build()
    pkg.load_library()


def _half_dims(d, Ns, i, h):
    s = d // Ns
    off = i * s
    ln = d - (Ns - 1) * s if i == Ns - 1 else s
    first = ln // 2
    return (off, first) if h == 0 else (off + first, ln - first)


def test_noalloc_kmeans_matches_the_index_build_twice_in_a_row():
    w = W.WORKLOADS[1]
    X = W.dataset(1)
    init = W.kmeans_init_ids(1, w.n, w.Ns, w.sqrtK)
    Xd = torch.from_numpy(X).cuda()
    iters = 5
    ix = pkg.suco_build_index(Xd, w.Ns, w.sqrtK, iters, init_ids=init)
    ex = pkg.suco_export_index(ix)
    pkg.suco_free(ix)
    K = w.sqrtK * w.sqrtK
    for (i, h) in ((0, 0), (5, 1)):  # two calls in a row share the fixed scratch
        off, ln = _half_dims(w.d, w.Ns, i, h)
        cent = torch.from_numpy(np.ascontiguousarray(X[init[i, h]][:, off:off + ln])).cuda()
        assign = pkg.suco_kmeans_noalloc(Xd, off, ln, cent, iters)
        torch.cuda.synchronize()
        np.testing.assert_allclose(cent.cpu().numpy(), ex["centroids"][i, h, :, :ln], rtol=1e-5, atol=1e-5)
        # the index's IMI cell of every point encodes the same assignment
        cell = np.empty(w.n, np.int64)
        off_i, perm_i = ex["cell_off"][i].astype(np.int64), ex["perm"][i]
        for c in range(K):
            cell[perm_i[off_i[c]:off_i[c + 1]]] = c
        expected = cell // w.sqrtK if h == 0 else cell % w.sqrtK
        np.testing.assert_array_equal(assign.cpu().numpy(), expected)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    Xd = torch.zeros((1000, 200), device="cuda")
    with pytest.raises(pkg.SucoError) as e:
        pkg.suco_kmeans_noalloc(Xd, 0, 129, torch.zeros((4, 129), device="cuda"), 1)
    assert e.value.code == -6
    with pytest.raises(pkg.SucoError) as e:
        pkg.suco_kmeans_noalloc(Xd, 0, 8, torch.zeros((257, 8), device="cuda"), 1)
    assert e.value.code == -6
