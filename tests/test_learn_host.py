"""Host-side logic of the learned ratios: grid labels and operating points (CPU only)."""
import math

import numpy as np

from paper_2411_14754_gb300 import learn as L

A, B = (0.01, 0.05, 0.1), (0.001, 0.004)


def _cost(n=1000, d=8, Ns=2):
    return np.array([[L.path_bytes(a, b, n, d, Ns) for b in B] for a in A])


def test_path_bytes_counts_ids_and_rows():
    assert L.path_bytes(0.05, 0.004, 1000, 8, 2) == 4 * 2 * 50 + 4 * 4 * 8


def test_full_labels_take_the_cheapest_point_with_recall_one():
    rec = np.zeros((3, 3, 2))
    rec[0] = 1.0                                   # easy: everything works
    rec[1, 2, 1] = 1.0                             # only the largest point
    rec[2] = 0.5                                   # never reaches 1: the largest point
    lab = L.labels_from_recalls(rec, 1000, 8, 2, alphas=A, betas=B, mode="full")
    c = _cost()
    ia, ib = np.unravel_index(np.argmin(c), c.shape)
    assert np.allclose(lab[0], [math.log(A[ia]), math.log(B[ib])])
    assert np.allclose(lab[1], [math.log(0.1), math.log(0.004)])
    assert np.allclose(lab[2], [math.log(0.1), math.log(0.004)])


def test_lagrange_labels_reach_the_target_at_least_cost():
    rng = np.random.default_rng(0)
    nq = 200
    # recall grows with alpha and beta at a per-query rate
    rate = rng.uniform(0.2, 5.0, nq)
    c = _cost()
    rec = 1.0 - np.exp(-rate[:, None, None] * c[None] / c.max() * 4)
    for target in (0.5, 0.8, 0.9):
        lab = L.labels_from_recalls(rec, 1000, 8, 2, alphas=A, betas=B, mode="lagrange", target=target)
        ia = np.array([A.index(a) for a in np.round(np.exp(lab[:, 0]), 6)])
        ib = np.array([B.index(b) for b in np.round(np.exp(lab[:, 1]), 6)])
        got = rec[np.arange(nq), ia, ib]
        assert got.mean() >= target - 1e-12
        # no single query can move to a cheaper point without the mean dropping below the target
        spent = c[ia, ib].sum()
        for q in range(nq):
            for ja in range(3):
                for jb in range(2):
                    if c[ja, jb] < c[ia[q], ib[q]]:
                        m = got.mean() - (got[q] - rec[q, ja, jb]) / nq
                        assert m < target or rec[q, ja, jb] < got[q] - 1e-12 or spent <= 0


def test_lagrange_with_an_unreachable_target_gives_every_query_its_best_recall():
    rec = np.full((4, 3, 2), 0.3)
    rec[:, 1, 0] = 0.6
    lab = L.labels_from_recalls(rec, 1000, 8, 2, alphas=A, betas=B, mode="lagrange", target=0.99)
    assert np.allclose(lab, [[math.log(0.05), math.log(0.001)]] * 4)


def test_cheapest_fixed_point():
    rm = np.array([[0.90, 0.94], [0.95, 0.97], [0.96, 0.99]])
    assert L.cheapest_fixed(rm, 1000, 8, 2, target=0.95, alphas=A, betas=B) == (0.05, 0.001)
    assert L.cheapest_fixed(rm, 1000, 8, 2, target=0.995, alphas=A, betas=B) == (0.1, 0.004)


def test_recall_rows():
    gt = np.array([[1, 2, 3, 4], [5, 6, 7, 8]])
    ids = np.array([[4, 3, 9, 1], [0, 0, 0, 0]])
    assert L.recall_rows(ids, gt).tolist() == [0.75, 0.0]
