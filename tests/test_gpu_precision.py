"""BF16 and FP8 coarse re-rank vs the reduced-precision oracle, through the C ABI.

The candidates come from the same bit-exact stages as the FP32 path; the coarse
pass reads the BF16 copy of the dataset, or its FP8 E4M3 copy with one scale
per subspace.  The survivors must be the R
candidates with the smallest (coarse distance, id): the GPU sums in FP32, the
oracle in FP64, so the two sets may differ only by candidates whose coarse
distance ties the R-th one within FP32 rounding.  The final top-k must be the
exact top-k of the GPU's own survivors, and with R >= C the result must equal
the FP32 path's bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2411_14754_gb300 as pkg
from oracle import precision_oracle as P
from paper_2411_14754_gb300 import workloads as W
from parity_util import check_coarse_against_oracle

pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2411_14754_gb300 import build
    build.build()
    pkg.load_library()


@pytest.fixture(scope="module")
def tiny():
    w = W.WORKLOADS[1]
    X = W.dataset(1)
    Q = W.queries(1)
    idx = oracle.build_index(X, w.Ns, w.sqrtK, w.kmeans_iters, W.kmeans_init_ids(1, w.n, w.Ns, w.sqrtK))
    return w, X, Q, idx


def gpu_index(X, idx_o):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    ix = pkg.suco_build_index_from_assignments(Xd, idx_o["Ns"], idx_o["sqrtK"], idx_o["centroids"], idx_o["assign"])
    pkg.suco_add_reduced_copies(ix)
    return ix


def check_bf16(X, idx_o, Q, k, alpha, beta, R, cluster_size=0, threads=0, prec="bf16"):
    ix = gpu_index(X, idx_o)
    scales = P.subspace_scales_e4m3(X, idx_o["Ns"]) if prec == "fp8" else None
    try:
        Qd = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
        out = pkg.suco_query_debug(ix, Qd, k, alpha, beta, cluster_size=cluster_size, threads=threads,
                                   want=("cands", "survivors"), precision=prec, exact_rerank=R)
        torch.cuda.synchronize()
        host = {kk: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for kk, v in out.items()}
    finally:
        pkg.suco_free(ix)
    T, C = host["T"], host["C"]
    for b in range(len(Q)):
        o = oracle.query(X, idx_o, Q[b], k, T, C, rank_precision=1, debug=True)
        check_coarse_against_oracle(X, Q[b], host["cands"][b], np.flatnonzero(host["survivors"][b]),
                                    host["ids"][b], host["dist"][b], o["cands"], k, R, prec, idx_o["Ns"], scales)
    return host


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("R", [10, 17, 32, 49])
def test_coarse_survivors_and_topk(tiny, R, prec):
    w, X, Q, idx = tiny
    check_bf16(X, idx, Q[:40], w.k, w.alpha, w.beta, R, prec=prec)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("cluster_size", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("threads", [256, 512, 1024])
def test_coarse_every_launch_shape(tiny, cluster_size, threads, prec):
    w, X, Q, idx = tiny
    check_bf16(X, idx, Q[:16], w.k, 0.1, 0.02, 37, cluster_size=cluster_size, threads=threads, prec=prec)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_coarse_with_all_candidates_surviving_equals_fp32(tiny, prec):
    w, X, Q, idx = tiny
    ix = gpu_index(X, idx)
    try:
        Qd = torch.from_numpy(Q).cuda()
        a = pkg.suco_query_batch(ix, Qd, w.k, w.alpha, w.beta)
        b = pkg.suco_query_batch(ix, Qd, w.k, w.alpha, w.beta, precision=prec, exact_rerank=50)
        torch.cuda.synchronize()
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    finally:
        pkg.suco_free(ix)


def test_bf16_exact_on_integer_data():
    # integer features <= 255 are exact in BF16: coarse == exact distance, the
    # survivors are the R nearest candidates, the result equals FP32's
    w = W.WORKLOADS[2]
    n = 20_000
    X = W.dataset(2, n=n)
    Q = W.queries(2, nq=24)
    idx = oracle.build_index(X, 8, 12, 5, W.kmeans_init_ids(2, n, 8, 12))
    host = check_bf16(X, idx, Q, 10, 0.05, 0.01, 64)
    ix = gpu_index(X, idx)
    try:
        a = pkg.suco_query_batch(ix, torch.from_numpy(Q).cuda(), 10, 0.05, 0.01)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(a[0].cpu().numpy(), host["ids"])
        np.testing.assert_array_equal(a[1].cpu().numpy(), host["dist"])
    finally:
        pkg.suco_free(ix)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_coarse_ragged_dimension_and_ties(prec):
    # d = 13 (rows padded to 16 BF16 values), many duplicate points (coarse ties broken by id)
    rng = np.random.default_rng(7)
    base = rng.integers(0, 4, size=(300, 13)).astype(np.float32) * 0.37
    X = np.repeat(base, 7, axis=0)[rng.permutation(2100)]
    Q = (rng.integers(0, 4, size=(12, 13)).astype(np.float32) * 0.37 + rng.normal(0, 0.01, (12, 13))).astype(np.float32)
    idx = oracle.build_index(X, 3, 4, 3, W.random_init_ids(9, X.shape[0], 3, 4))
    check_bf16(X, idx, Q, 5, 0.3, 0.1, 23, prec=prec)


def test_reduced_precision_needs_its_copy(tiny):
    w, X, Q, idx = tiny
    Xd = torch.from_numpy(X).cuda()
    ix = pkg.suco_build_index_from_assignments(Xd, idx["Ns"], idx["sqrtK"], idx["centroids"], idx["assign"])
    try:
        with pytest.raises(pkg.SucoError) as e:
            pkg.suco_query_batch(ix, torch.from_numpy(Q).cuda(), w.k, w.alpha, w.beta, precision="bf16")
        assert e.value.code == -5
        with pytest.raises(pkg.SucoError) as e:
            pkg.suco_query_batch(ix, torch.from_numpy(Q).cuda(), w.k, w.alpha, w.beta, precision="fp8")
        assert e.value.code == -5
        with pytest.raises(pkg.SucoError):
            pkg.suco_query_batch(ix, torch.from_numpy(Q).cuda(), w.k, w.alpha, w.beta, precision=7)
    finally:
        pkg.suco_free(ix)


def test_fp8_codes_match_the_oracle_on_a_subspace_with_a_large_range():
    # one subspace spans 1000x the range of the others: its own scale keeps its
    # codes informative; the coarse pass still selects the oracle's survivors
    rng = np.random.default_rng(9)
    X = np.abs(rng.standard_normal((3000, 24))).astype(np.float32)
    X[:, 16:] *= 1000.0
    Q = np.abs(rng.standard_normal((16, 24))).astype(np.float32)
    Q[:, 16:] *= 1000.0
    idx = oracle.build_index(X, 3, 6, 3, W.random_init_ids(10, 3000, 3, 6))
    check_bf16(X, idx, Q, 7, 0.2, 0.05, 31, prec="fp8")
