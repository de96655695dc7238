"""GPU index construction (Algorithm 2) vs the CPU oracle, through the C ABI."""
import numpy as np
import pytest
import torch
from scipy.spatial.distance import cdist

import oracle
import paper_2411_14754_gb300 as pkg
from paper_2411_14754_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2411_14754_gb300 import build
    build.build()
    pkg.load_library()


def _cells_from_csr(off, perm, n, K):
    cell = np.empty(n, np.int64)
    for c in range(K):
        cell[perm[off[c]:off[c + 1]]] = c
    return cell


@pytest.mark.parametrize("n,d,Ns,sk", [(10_000, 128, 8, 10), (1001, 13, 3, 5), (4000, 64, 16, 33), (300, 8, 2, 20),
                                      (100, 4, 1, 10), (70_000, 8, 1, 256), (2048 * 3 + 1, 16, 2, 17)])
def test_imi_from_assignments_is_bit_exact(n, d, Ns, sk):
    # one radix pass for K <= 256, two above it (K = 65536 uses both digits
    # whole); tiles of 2048 keys, whole and ragged
    X = W.random_data(n + d, n, d)
    rng = np.random.default_rng(n)
    assign = rng.integers(0, sk, size=(Ns, 2, n)).astype(np.int32)
    hm = oracle.hmax(d, Ns)
    cents = rng.random((Ns, 2, sk, hm)).astype(np.float32)
    ref = oracle.index_from_parts(Ns, sk, cents, assign)
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).cuda(), Ns, sk, cents, assign)
    ex = pkg.suco_export_index(ix)
    pkg.suco_free(ix)
    np.testing.assert_array_equal(ex["cell_off"].astype(np.int64), ref["cell_off"])
    np.testing.assert_array_equal(ex["perm"].astype(np.int64), ref["perm"])
    for i in range(Ns):
        for h in range(2):
            off, ln = oracle.half_dims(d, Ns, i, h)
            np.testing.assert_array_equal(ex["centroids"][i, h, :, :ln], cents[i, h, :, :ln])


def test_kmeans_one_iteration_matches_oracle():
    w = W.WORKLOADS[1]
    X = W.dataset(1)
    init = W.kmeans_init_ids(1, w.n, w.Ns, w.sqrtK)
    ix = pkg.suco_build_index(torch.from_numpy(X).cuda(), w.Ns, w.sqrtK, 1, init_ids=init)
    ex = pkg.suco_export_index(ix)
    pkg.suco_free(ix)
    ref = oracle.build_index(X, w.Ns, w.sqrtK, 1, init)
    mism = 0
    for i in range(w.Ns):
        for h in range(2):
            off, ln = oracle.half_dims(w.d, w.Ns, i, h)
            g = ex["centroids"][i, h, :, :ln].astype(np.float64)
            o = ref["centroids"][i, h, :, :ln].astype(np.float64)
            np.testing.assert_allclose(g, o, rtol=1e-5, atol=1e-5)
        # final assignment: the cells of the GPU IMI vs argmin against the GPU's own centroids (FP64)
        cell = _cells_from_csr(ex["cell_off"][i].astype(np.int64), ex["perm"][i], w.n, w.sqrtK ** 2)
        for h in range(2):
            off, ln = oracle.half_dims(w.d, w.Ns, i, h)
            dd = cdist(X[:, off:off + ln].astype(np.float64), ex["centroids"][i, h, :, :ln].astype(np.float64),
                       "sqeuclidean")
            best = np.argmin(dd, axis=1)
            got = cell // w.sqrtK if h == 0 else cell % w.sqrtK
            bad = np.where(got != best)[0]
            # a different choice is allowed only where two centroids tie within FP32 rounding
            for p in bad:
                assert abs(dd[p, got[p]] - dd[p, best[p]]) <= 1e-5 * max(dd[p, best[p]], 1.0)
            mism += len(bad)
    assert mism <= 10


@pytest.mark.parametrize("d,Ns,metric", [(13, 2, "l2"), (48, 2, "l2"), (50, 2, "l2"), (120, 2, "l2"), (80, 1, "l2"),
                                         (50, 2, "l1"), (120, 2, "l1"), (80, 1, "l1")])
def test_kmeans_iteration_matches_oracle_for_each_half_length(d, Ns, metric):
    # halves of 3-4 dims (the assignment kernel's 8-wide rows), 12-13 (16-wide),
    # 30 (32-wide) and 40 (the any-length kernel), under both metrics: one
    # Lloyd iteration from given points, then the final assignment
    n, sk = 3000, 8
    X = W.random_data(7 + d, n, d)
    rng = np.random.default_rng(d)
    init = np.stack([np.stack([rng.choice(n, sk, replace=False) for _ in range(2)]) for _ in range(Ns)])
    m = oracle.METRIC_L1 if metric == "l1" else 0
    ix = pkg.suco_build_index(torch.from_numpy(X).cuda(), Ns, sk, 1, init_ids=init, metric=metric)
    ex = pkg.suco_export_index(ix)
    pkg.suco_free(ix)
    ref = oracle.build_index(X, Ns, sk, 1, init, metric=m)
    kind = "cityblock" if m else "sqeuclidean"
    for i in range(Ns):
        cell = _cells_from_csr(ex["cell_off"][i].astype(np.int64), ex["perm"][i], n, sk * sk)
        for h in range(2):
            off, ln = oracle.half_dims(d, Ns, i, h)
            g = ex["centroids"][i, h, :, :ln].astype(np.float64)
            np.testing.assert_allclose(g, ref["centroids"][i, h, :, :ln], rtol=1e-5, atol=1e-5)
            dd = cdist(X[:, off:off + ln].astype(np.float64), g, kind)
            got = cell // sk if h == 0 else cell % sk
            best = dd.min(axis=1)
            np.testing.assert_allclose(dd[np.arange(n), got], best, rtol=1e-5, atol=1e-6)


def test_kmeans_converges_on_separated_blobs():
    rng = np.random.default_rng(3)
    centres = rng.uniform(0, 1000, size=(5, 4))
    lab = rng.integers(0, 5, size=5000)
    X = (centres[lab] + rng.normal(0, 1, size=(5000, 4))).astype(np.float32)
    init = np.empty((1, 2, 5), np.int64)
    for h in range(2):
        init[0, h] = [int(np.where(lab == c)[0][0]) for c in range(5)]
    ix = pkg.suco_build_index(torch.from_numpy(X).cuda(), 1, 5, 20, init_ids=init)
    ex = pkg.suco_export_index(ix)
    pkg.suco_free(ix)
    ref = oracle.build_index(X, 1, 5, 20, init)
    np.testing.assert_allclose(ex["centroids"], ref["centroids"], rtol=1e-5, atol=1e-4)
    np.testing.assert_array_equal(ex["cell_off"].astype(np.int64), ref["cell_off"])
    np.testing.assert_array_equal(ex["perm"].astype(np.int64), ref["perm"])


def test_build_is_deterministic_and_seeded():
    X = torch.from_numpy(W.dataset(1, n=5000)).cuda()
    a = pkg.suco_export_index(pkg.suco_build_index(X, 8, 10, 5, seed=7))
    b = pkg.suco_export_index(pkg.suco_build_index(X, 8, 10, 5, seed=7))
    c = pkg.suco_export_index(pkg.suco_build_index(X, 8, 10, 5, seed=8))
    for key in ("centroids", "cell_off", "perm"):
        np.testing.assert_array_equal(a[key], b[key])
    assert not np.array_equal(a["centroids"], c["centroids"])


def test_build_argument_errors():
    X = torch.zeros((100, 16), device="cuda")
    for args in ((0, 4), (9, 4), (8, 257), (8, 101)):   # Ns < 1, d < 2*Ns, sqrtK > 256, sqrtK > n
        with pytest.raises(pkg.SucoError) as e:
            pkg.suco_build_index(X, args[0], args[1], 2)
        assert e.value.code == -1
    with pytest.raises(pkg.SucoError):
        pkg.suco_build_index(X, 2, 4, 2, init_ids=np.zeros((2, 2, 4), np.int64))   # repeated init ids
