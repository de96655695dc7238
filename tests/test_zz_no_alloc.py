"""suco_kmeans_noalloc: K-means on one column range with no device allocation in
the library (its scratch is a fixed array defined in the library).

Callers that cannot allocate device memory when they run the step use this
entry point: a process whose device memory is already handed to its own
allocator, or a caller under a latency budget that rules out cudaMalloc.  Its
results are checked against the CPU oracle's Lloyd iterations (FP64), on a
narrow shape whose sums fit shared memory and on the largest shape the fixed
array takes (k = 256 centroids, 128 columns), whose sums go through the array
in global memory; the calls run small, large, small, so that a later call
finds the array holding a wider earlier call's contents.  This file is
collected last so that, if it fails, every other test has already run.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2411_14754_gb300 as pkg
from paper_2411_14754_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# centroids: FP32 means of fixed-point sums (at most two roundings) against the
# oracle's FP64 means; assignments: exact, except where two centroids are at
# the same distance within FP32 error
CENT_RTOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2411_14754_gb300 import build
    build.build()
    pkg.load_library()


def _check_against_oracle(X, Xd, off, ln, init, iters):
    cent_o, _ = oracle.kmeans(X, off, ln, len(init), iters, init)
    cent = torch.from_numpy(np.ascontiguousarray(X[init][:, off:off + ln])).cuda()
    assign = pkg.suco_kmeans_noalloc(Xd, off, ln, cent, iters)
    torch.cuda.synchronize()
    cg = cent.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(cg, cent_o, rtol=CENT_RTOL, atol=1e-6 * np.abs(cent_o).max())
    # the final assignment: the nearest of the oracle's centroids (as stored, FP32)
    expected = oracle.assign_nearest(X, off, ln, cent_o.astype(np.float32))
    got = assign.cpu().numpy()
    bad = np.flatnonzero(got != expected)
    if len(bad):
        xs = X[bad][:, off:off + ln].astype(np.float64)
        c32 = cent_o.astype(np.float32).astype(np.float64)
        dg = ((xs - c32[got[bad]]) ** 2).sum(1)
        de = ((xs - c32[expected[bad]]) ** 2).sum(1)
        np.testing.assert_allclose(dg, de, rtol=1e-5)
    assert len(bad) <= max(1, len(X) // 1000)


def test_noalloc_kmeans_matches_the_oracle_small_large_small():
    w = W.WORKLOADS[1]
    X = W.dataset(1)
    Xd = torch.from_numpy(X).cuda()
    small_init = np.random.default_rng(62).choice(w.n, size=50, replace=False)
    # integer data for the wide shape: the first assignment (against data rows)
    # is exact in FP32, so one Lloyd step leaves no room for a diverging path
    Xi = W.random_data(63, w.n, w.d, kind="int")
    Xid = torch.from_numpy(Xi).cuda()
    large_init = np.random.default_rng(64).choice(w.n, size=256, replace=False)
    _check_against_oracle(X, Xd, 8, 8, small_init, 4)          # sums in shared memory
    _check_against_oracle(Xi, Xid, 0, 128, large_init, 1)      # k*dim_len*8 bytes exceed shared memory
    _check_against_oracle(X, Xd, 8, 8, small_init, 4)          # the array now holds the wide call's sums


def test_noalloc_two_calls_in_a_row_agree_with_the_index_build():
    # two calls in a row share the fixed array; each equals the K-means that
    # suco_build_index runs with allocated scratch (same kernels, same order)
    w = W.WORKLOADS[1]
    X = W.dataset(1)
    init = W.kmeans_init_ids(1, w.n, w.Ns, w.sqrtK)
    Xd = torch.from_numpy(X).cuda()
    iters = 5
    ix = pkg.suco_build_index(Xd, w.Ns, w.sqrtK, iters, init_ids=init)
    ex = pkg.suco_export_index(ix)
    pkg.suco_free(ix)
    K = w.sqrtK * w.sqrtK
    for (i, h) in ((0, 0), (5, 1)):
        off, ln = oracle.half_dims(w.d, w.Ns, i, h)
        cent = torch.from_numpy(np.ascontiguousarray(X[init[i, h]][:, off:off + ln])).cuda()
        assign = pkg.suco_kmeans_noalloc(Xd, off, ln, cent, iters)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(cent.cpu().numpy(), ex["centroids"][i, h, :, :ln])
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


def test_noalloc_refuses_an_output_it_would_overrun():
    Xd = torch.zeros((1000, 16), device="cuda")
    cent = torch.zeros((4, 8), device="cuda")
    with pytest.raises(ValueError):
        pkg.suco_kmeans_noalloc(Xd, 0, 8, cent, 1, assign=torch.empty(999, dtype=torch.int32, device="cuda"))
    with pytest.raises(TypeError):
        pkg.suco_kmeans_noalloc(Xd, 0, 8, cent, 1, assign=torch.empty(1000, dtype=torch.int16, device="cuda"))
