"""BF16 and FP8 tensor-core ranking (tcgen05) vs the oracle, through the C ABI.

The kernel rounds the query and the centroids to BF16 (or codes them as E4M3
with one scale per subspace) and forms |q|^2 - 2<q,c> + |c|^2 from
tensor-core inner products with FP32 accumulation.
Its tables must match the FP64 squared distances of the same rounded vectors
within the FP32 error of that expression; every later stage (cell activation,
SC-scores, candidates, top-k) must then be exactly what the oracle computes
from the GPU's own tables.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2411_14754_gb300 as pkg
from oracle import precision_oracle as P
from paper_2411_14754_gb300 import workloads as W
from parity_util import assert_topk_matches

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2411_14754_gb300 import build
    build.build()
    pkg.load_library()


def gpu_index(X, idx):
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(np.ascontiguousarray(X)).cuda(), idx["Ns"],
                                               idx["sqrtK"], idx["centroids"], idx["assign"])
    pkg.suco_add_reduced_copies(ix)
    return ix


def check(X, idx, Q, k, alpha, beta, sample=None, rank="bf16", **kw):
    ix = gpu_index(X, idx)
    try:
        Qd = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
        out = pkg.suco_query_debug(ix, Qd, k, alpha, beta, rank_precision=rank, **kw)
        full = pkg.suco_query_batch(ix, Qd, k, alpha, beta, rank_precision=rank, **kw)
        torch.cuda.synchronize()
        assert pkg.suco_read_status(ix) == 0
        host = {kk: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for kk, v in out.items()}
    finally:
        pkg.suco_free(ix)
    np.testing.assert_array_equal(full[0].cpu().numpy(), host["ids"])
    T, C = host["T"], host["C"]
    d = X.shape[1]
    scales = P.subspace_scales_e4m3(X, idx["Ns"]) if rank == "fp8" else None
    worst = 0.0
    for b in (range(len(Q)) if sample is None else sample):
        if rank == "fp8":
            ref, norms = P.fp8_centroid_tables(idx, Q[b], scales)
        else:
            ref, norms = P.bf16_centroid_tables(idx, Q[b])
        L = np.array([[oracle.half_dims(d, idx["Ns"], i, h)[1] for h in range(2)] for i in range(idx["Ns"])])
        tol = (4.0 * L[:, :, None] + 64.0) * U * norms
        got = host["dtab"][b].astype(np.float64)
        worst = max(worst, float((np.abs(got - ref) / np.maximum(norms * U, 1e-300)).max()))
        assert (np.abs(got - ref) <= tol).all(), np.abs(got - ref).max()
        o = oracle.query_from_tables(X, idx, Q[b], k, T, C, got)
        np.testing.assert_array_equal(host["t_eff"][b], o["teff"])
        np.testing.assert_array_equal(host["activated"][b], o["activated"])
        np.testing.assert_array_equal(host["scores"][b].astype(np.int32), o["scores"])
        assert sorted(host["cands"][b].tolist()) == sorted(o["cands"].tolist())
        assert_topk_matches(X, Q[b], host["ids"][b], host["dist"][b], o["ids"], o["dist"])
    print(f"\n{rank} ranking tables: largest |error| / (u * (|q|^2 + |c|^2)) = {worst:.1f}")


@pytest.fixture(scope="module")
def tiny():
    w = W.WORKLOADS[1]
    X = W.dataset(1)
    idx = oracle.build_index(X, w.Ns, w.sqrtK, w.kmeans_iters, W.kmeans_init_ids(1, w.n, w.Ns, w.sqrtK))
    return w, X, idx


RANKS = ["bf16", "fp8"]


@pytest.mark.parametrize("rank", RANKS)
def test_tiny_workload_tables_and_stages(tiny, rank):
    w, X, idx = tiny
    check(X, idx, W.queries(1), w.k, w.alpha, w.beta, rank=rank)


@pytest.mark.parametrize("rank", RANKS)
def test_two_launch_chunks_and_a_ragged_tail(tiny, rank):
    # 4096 queries per tensor-core launch: rows from both chunks and the tail tile
    w, X, idx = tiny
    Q = W.queries(1, nq=4096 + 301)
    check(X, idx, Q, w.k, w.alpha, w.beta, sample=[0, 127, 128, 4095, 4096, 4200, 4396], rank=rank)


@pytest.mark.parametrize("rank", RANKS)
@pytest.mark.parametrize("n,d,Ns,sk", [(3000, 13, 3, 16), (4000, 64, 16, 33), (20000, 24, 2, 256), (600, 8, 4, 1),
                                       (5000, 120, 2, 40)])
def test_shapes(n, d, Ns, sk, rank):
    # ragged halves, many subspaces, the widest codebook (N = 256), one
    # centroid, halves of 30 (two FP8 MMAs along K for BF16's four)
    X = W.random_data(21, n, d, "gauss") * np.float32(3.0)
    Q = W.random_data(22, 40, d, "gauss") * np.float32(3.0)
    idx = oracle.build_index(X, Ns, sk, 2, W.random_init_ids(23, n, Ns, sk))
    check(X, idx, Q, 5, 0.05, 0.02, rank=rank)


def test_fp8_ranking_on_the_precision_workload_shape():
    # GIST-like values (non-negative, 30 % zeros), d = 960, Ns = 16, sqrtK = 64
    X = W.dataset(3, n=20_000)
    Q = W.queries(3, nq=64)
    idx = oracle.build_index(X, 16, 64, 2, W.kmeans_init_ids(3, 20_000, 16, 64))
    check(X, idx, Q, 10, 0.03, 0.005, sample=[0, 17, 63], rank="fp8")


def test_fp8_ranking_needs_the_fp8_scales(tiny):
    w, X, idx = tiny
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).cuda(), w.Ns, w.sqrtK, idx["centroids"],
                                               idx["assign"])
    try:
        pkg.suco_add_reduced_copies(ix, bf16=False, rank_bf16=True, fp8=False)
        with pytest.raises(pkg.SucoError) as e:
            pkg.suco_query_batch(ix, torch.from_numpy(W.queries(1)).cuda(), w.k, w.alpha, w.beta,
                                 rank_precision="fp8")
        assert e.value.code == -5
    finally:
        pkg.suco_free(ix)


def test_needs_the_workspace(tiny):
    w, X, idx = tiny
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).cuda(), w.Ns, w.sqrtK, idx["centroids"],
                                               idx["assign"])
    try:
        with pytest.raises(pkg.SucoError) as e:
            pkg.suco_query_batch(ix, torch.from_numpy(W.queries(1)).cuda(), w.k, w.alpha, w.beta,
                                 rank_precision="bf16")
        assert e.value.code == -5
    finally:
        pkg.suco_free(ix)
