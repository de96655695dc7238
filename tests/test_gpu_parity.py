"""GPU query path vs the CPU oracle, element by element, through the C ABI.

Both sides use the same index (the oracle's, loaded with
suco_build_index_from_assignments) and the same seeded inputs.  The oracle takes
the cell-ranking decisions in the kernel's FP32 arithmetic, so the centroid
distances, retrieved cells, SC-scores and candidate sets must be bit-exact; the
re-rank distances must agree within 1e-5 relative (FP32 vs FP64).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2411_14754_gb300 as pkg
from paper_2411_14754_gb300 import workloads as W
from parity_util import check_query_against_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2411_14754_gb300 import build
    build.build()
    pkg.load_library()


def run(X, idx_o, Q, k, alpha, beta, cluster_size=0, threads=0, stages=True, want=None, sample=None, flags=0,
        id_passes=0):
    dev = torch.device("cuda")
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).to(dev)
    ix = pkg.suco_build_index_from_assignments(Xd, idx_o["Ns"], idx_o["sqrtK"], idx_o["centroids"], idx_o["assign"])
    try:
        want = want or (("t_eff", "activated", "dtab", "scores", "cands") if stages else ())
        out = pkg.suco_query_debug(ix, Qd, k, alpha, beta, cluster_size=cluster_size, threads=threads, want=want,
                                   flags=flags, id_passes=id_passes)
        torch.cuda.synchronize()
        host = {kk: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for kk, v in out.items()}
    finally:
        pkg.suco_free(ix)
    T, C = host["T"], host["C"]
    assert T == oracle.collision_threshold(alpha, X.shape[0])
    assert C == oracle.candidate_count(beta, X.shape[0], k)
    rows = range(len(Q)) if sample is None else sample
    for b in rows:
        check_query_against_oracle(X, idx_o, Q[b], host, b, k, T, C, stages=stages)
    return host


@pytest.fixture(scope="module")
def tiny():
    w = W.WORKLOADS[1]
    X = W.dataset(1)
    Q = W.queries(1)
    idx = oracle.build_index(X, w.Ns, w.sqrtK, w.kmeans_iters, W.kmeans_init_ids(1, w.n, w.Ns, w.sqrtK))
    return w, X, Q, idx


def test_tiny_workload_all_queries(tiny):
    w, X, Q, idx = tiny
    run(X, idx, Q, w.k, w.alpha, w.beta)


@pytest.mark.parametrize("cluster_size", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("flags", [0, 1])
@pytest.mark.parametrize("threads", [256, 512, 1024])
def test_tiny_workload_every_launch_shape(tiny, cluster_size, threads, flags):
    w, X, Q, idx = tiny
    run(X, idx, Q[:24], w.k, w.alpha, w.beta, cluster_size=cluster_size, threads=threads, flags=flags)


@pytest.mark.parametrize("alpha,beta,k", [(0.01, 0.001, 10), (0.2, 0.02, 50), (1.0, 0.005, 10), (0.05, 1.0, 7),
                                          (0.003, 0.0005, 256), (1.0, 1.0, 20)])
def test_tiny_workload_alpha_beta_k(tiny, alpha, beta, k):
    w, X, Q, idx = tiny
    host = run(X, idx, Q[:10], k, alpha, beta)
    if alpha == 1.0:
        assert (host["scores"] == w.Ns).all()


def _idx(X, Ns, sk, iters, seed):
    return oracle.build_index(X, Ns, sk, iters, W.random_init_ids(seed, X.shape[0], Ns, sk))


def test_ragged_sizes_and_odd_dimension():
    # n not a multiple of 4 or 16, d not a multiple of 4, last subspace longer (Definition 3)
    X = W.random_data(1, 1001, 13)
    Q = W.random_data(2, 9, 13)
    run(X, _idx(X, 3, 5, 4, 3), Q, 10, 0.07, 0.02)


def test_many_empty_cells():
    X = W.random_data(3, 500, 16)
    Q = W.random_data(4, 6, 16)
    run(X, _idx(X, 4, 40, 3, 5), Q, 10, 0.1, 0.05)


def test_one_giant_cell_and_duplicate_points():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((3000, 24)).astype(np.float32)
    X[:2500] = X[0]                       # one cell holds most points; distances tie
    Q = np.concatenate([X[:2], rng.standard_normal((4, 24)).astype(np.float32)])
    run(X, _idx(X, 4, 6, 3, 7), Q, 12, 0.05, 0.01)


def test_all_points_in_one_cell_all_scores_tied():
    X = np.ones((777, 8), np.float32)
    Q = W.random_data(8, 3, 8)
    host = run(X, _idx(X, 2, 4, 2, 9), Q, 5, 0.05, 0.01)
    assert (host["scores"] == 2).all()
    # every distance ties: the lowest ids win
    assert host["ids"][0].tolist() == list(range(5))


def test_fewer_points_than_k():
    X = W.random_data(10, 5, 8)
    Q = W.random_data(11, 3, 8)
    host = run(X, _idx(X, 2, 2, 1, 12), Q, 10, 0.5, 0.5)
    assert (host["ids"][:, 5:] == -1).all() and np.isinf(host["dist"][:, 5:]).all()


@pytest.mark.parametrize("Ns,d,sk", [(1, 4, 3), (16, 64, 8), (32, 64, 4), (8, 96, 1), (2, 16, 256)])
def test_subspace_and_codebook_extremes(Ns, d, sk):
    n = max(3000, sk * 4)
    X = W.random_data(13, n, d, kind="uniform")
    Q = W.random_data(14, 5, d, kind="uniform")
    run(X, _idx(X, Ns, sk, 2, 15), Q, 10, 0.05, 0.01)


def test_exact_integer_data_matches_fp64_ranking():
    # small integers: FP32 arithmetic is exact, so the GPU must also match the
    # oracle run in the paper's FP64 arithmetic
    X = W.random_data(16, 4000, 32, kind="int")
    Q = W.random_data(17, 8, 32, kind="int")
    idx = _idx(X, 4, 8, 0, 18)
    host = run(X, idx, Q, 10, 0.05, 0.01)
    for b in range(len(Q)):
        o = oracle.query(X, idx, Q[b], 10, host["T"], host["C"], rank_precision=0)
        np.testing.assert_array_equal(host["scores"][b].astype(np.int32), o["scores"])


def test_single_query_and_empty_batch():
    X = W.dataset(1, n=2000)
    Q = W.queries(1, nq=1)
    idx = _idx(X, 8, 5, 3, 19)
    run(X, idx, Q, 10, 0.05, 0.005)
    dev = torch.device("cuda")
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).to(dev), 8, 5, idx["centroids"], idx["assign"])
    ids, dist = pkg.suco_query_batch(ix, torch.empty((0, X.shape[1]), device=dev), 10, 0.05, 0.005)
    assert ids.shape == (0, 10)
    pkg.suco_free(ix)


def test_query_batch_equals_debug_path(tiny):
    w, X, Q, idx = tiny
    dev = torch.device("cuda")
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).to(dev), w.Ns, w.sqrtK, idx["centroids"],
                                               idx["assign"])
    Qd = torch.from_numpy(Q).to(dev)
    a_ids, a_d = pkg.suco_query_batch(ix, Qd, w.k, w.alpha, w.beta)
    b = pkg.suco_query_debug(ix, Qd, w.k, w.alpha, w.beta, want=())
    a2_ids, a2_d = pkg.suco_query_batch(ix, Qd, w.k, w.alpha, w.beta)
    torch.cuda.synchronize()
    assert torch.equal(a_ids, b["ids"]) and torch.equal(a_d, b["dist"])
    assert torch.equal(a_ids, a2_ids) and torch.equal(a_d, a2_d)      # deterministic
    pkg.suco_free(ix)


def test_argument_errors_on_device(tiny):
    w, X, Q, idx = tiny
    dev = torch.device("cuda")
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).to(dev), w.Ns, w.sqrtK, idx["centroids"],
                                               idx["assign"])
    Qd = torch.from_numpy(Q[:2]).to(dev)
    for kw in (dict(k=0, alpha=0.05, beta=0.01), dict(k=10, alpha=0.0, beta=0.01), dict(k=10, alpha=0.05, beta=1.5),
               dict(k=10, alpha=0.05, beta=0.01, cluster_size=3), dict(k=10, alpha=0.05, beta=0.01, threads=384),
               dict(k=257, alpha=0.05, beta=0.01)):
        with pytest.raises(pkg.SucoError) as e:
            pkg.suco_query_batch(ix, Qd, **kw)
        assert e.value.code == -1
    bad = idx["assign"].copy()
    bad[0, 0, 0] = w.sqrtK
    with pytest.raises(pkg.SucoError):
        pkg.suco_build_index_from_assignments(torch.from_numpy(X).to(dev), w.Ns, w.sqrtK, idx["centroids"], bad)
    pkg.suco_free(ix)


def test_score_array_too_large_is_reported():
    # forced into one pass, the SC-score counters of 8M ids (Ns = 32: two nibble
    # sets and two one-bit planes, 10 bits per id) do not fit 16 CTAs
    n = 8_000_000
    dev = torch.device("cuda")
    X = torch.zeros((n, 64), device=dev)
    ix = pkg.suco_build_index(X, 32, 1, 0)
    del X
    q = torch.zeros((1, 64), device=dev)
    with pytest.raises(pkg.SucoError) as e:
        pkg.suco_query_batch(ix, q, 10, 0.01, 0.001, id_passes=1)
    assert e.value.code == -6
    # the automatic launch takes several passes: every point sits on the query
    # and scores Ns, so the answer is the 10 lowest ids at distance 0
    ids, dist = pkg.suco_query_batch(ix, q, 10, 0.01, 0.001)
    torch.cuda.synchronize()
    assert ids.cpu().tolist() == [list(range(10))]
    assert dist.abs().max().item() == 0.0
    pkg.suco_free(ix)


def test_per_query_k_alpha_beta(tiny):
    # a mixed batch: every query has its own k, alpha and beta (device arrays); the
    # scalar beta bounds the per-query values
    w, X, Q, idx = tiny
    rng = np.random.default_rng(77)
    nq = 48
    ks = rng.choice([1, 10, 37], nq).astype(np.int32)
    al = rng.choice([0.01, 0.03, 0.05, 0.2], nq).astype(np.float32)
    be = rng.choice([0.001, 0.003, 0.005, 0.02, 0.5], nq).astype(np.float32)
    kmax, beta_bound = 37, 0.02
    dev = torch.device("cuda")
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).to(dev), w.Ns, w.sqrtK, idx["centroids"],
                                               idx["assign"])
    try:
        out = pkg.suco_query_debug(ix, torch.from_numpy(Q[:nq]).to(dev), kmax, 0.05, beta_bound,
                                   k_per_query=torch.from_numpy(ks).to(dev),
                                   alpha_per_query=torch.from_numpy(al).to(dev),
                                   beta_per_query=torch.from_numpy(be).to(dev))
        torch.cuda.synchronize()
        host = {kk: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for kk, v in out.items()}
    finally:
        pkg.suco_free(ix)
    n = X.shape[0]
    for b in range(nq):
        kb = int(ks[b])
        T = oracle.collision_threshold(float(al[b]), n)
        C = oracle.candidate_count(min(float(be[b]), beta_bound), n, kb)
        o = oracle.query(X, idx, Q[b], kb, T, C, rank_precision=1)
        np.testing.assert_array_equal(host["t_eff"][b], o["teff"])
        np.testing.assert_array_equal(host["scores"][b].astype(np.int32), o["scores"])
        assert sorted(host["cands"][b][:C].tolist()) == sorted(o["cands"].tolist())
        from parity_util import assert_topk_matches
        assert_topk_matches(X, Q[b], host["ids"][b][:kb], host["dist"][b][:kb], o["ids"], o["dist"])
        assert (host["ids"][b][kb:] == -1).all() and np.isinf(host["dist"][b][kb:]).all()


def test_one_cluster_per_query_flag(tiny):
    w, X, Q, idx = tiny
    dev = torch.device("cuda")
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).to(dev), w.Ns, w.sqrtK, idx["centroids"],
                                               idx["assign"])
    Qd = torch.from_numpy(Q).to(dev)
    a = pkg.suco_query_batch(ix, Qd, w.k, w.alpha, w.beta)
    b = pkg.suco_query_batch(ix, Qd, w.k, w.alpha, w.beta, flags=pkg.suco.QUERY_ONE_CLUSTER_PER_QUERY)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    pkg.suco_free(ix)
    host = run(X, idx, Q[:16], w.k, w.alpha, w.beta)  # persistent path against the oracle already covered
    assert host["ids"].shape == (16, w.k)


def test_autotune_picks_a_shape_with_identical_results(tiny):
    w, X, Q, idx = tiny
    dev = torch.device("cuda")
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).to(dev), w.Ns, w.sqrtK, idx["centroids"],
                                               idx["assign"])
    Qd = torch.from_numpy(Q).to(dev)
    ref = pkg.suco_query_batch(ix, Qd, w.k, w.alpha, w.beta, cluster_size=1, threads=512)
    cl, nt = pkg.suco_autotune(ix, Qd, w.k, w.alpha, w.beta)
    assert cl in (1, 2, 4, 8, 16) and nt in (256, 512, 1024)
    got = pkg.suco_query_batch(ix, Qd, w.k, w.alpha, w.beta)
    torch.cuda.synchronize()
    assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1])
    pkg.suco_free(ix)


def test_query_replays_from_a_cuda_graph(tiny):
    w, X, Q, idx = tiny
    dev = torch.device("cuda")
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).to(dev), w.Ns, w.sqrtK, idx["centroids"],
                                               idx["assign"])
    Qd = torch.from_numpy(Q[:32]).to(dev)
    ids = torch.empty((32, w.k), dtype=torch.int32, device=dev)
    dist = torch.empty((32, w.k), dtype=torch.float32, device=dev)
    ref = pkg.suco_query_batch(ix, Qd, w.k, w.alpha, w.beta)  # first call outside capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pkg.suco_query_batch(ix, Qd, w.k, w.alpha, w.beta, out_ids=ids, out_dist=dist, stream=s)
    for rep in range(3):
        ids.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(ids, ref[0]) and torch.equal(dist, ref[1])
    # replay on new inputs written into the captured buffer
    Qd.copy_(torch.from_numpy(Q[32:64]).to(dev))
    g.replay()
    ref2 = pkg.suco_query_batch(ix, Qd, w.k, w.alpha, w.beta)
    torch.cuda.synchronize()
    assert torch.equal(ids, ref2[0])
    pkg.suco_free(ix)


def test_work_counter_answers_every_query_once_across_calls_and_replays(tiny):
    # many more queries than resident clusters, of very uneven cost: the
    # persistent launch hands queries out through the index's work counters,
    # which must cover every query once per call and be back at zero for the
    # next call (plain calls, calls on a second stream, graph replays)
    w, X, Q, idx = tiny
    dev = torch.device("cuda")
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).to(dev), w.Ns, w.sqrtK, idx["centroids"],
                                               idx["assign"])
    nq = 3000
    Qd = torch.from_numpy(W.queries(1, nq=nq)).to(dev)
    rng = np.random.default_rng(5)
    al = torch.from_numpy(rng.choice([0.005, 0.05, 0.6], nq, p=[0.6, 0.3, 0.1]).astype(np.float32)).to(dev)
    kw = dict(alpha_per_query=al)
    ref = pkg.suco_query_batch(ix, Qd, w.k, 0.05, w.beta, flags=pkg.suco.QUERY_ONE_CLUSTER_PER_QUERY, **kw)
    for _ in range(3):
        got = pkg.suco_query_batch(ix, Qd, w.k, 0.05, w.beta, **kw)
        torch.cuda.synchronize()
        assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    ids = torch.empty((nq, w.k), dtype=torch.int32, device=dev)
    dist = torch.empty((nq, w.k), dtype=torch.float32, device=dev)
    with torch.cuda.stream(s):
        pkg.suco_query_batch(ix, Qd, w.k, 0.05, w.beta, out_ids=ids, out_dist=dist, stream=s, **kw)
    s.synchronize()
    assert torch.equal(ids, ref[0])
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pkg.suco_query_batch(ix, Qd, w.k, 0.05, w.beta, out_ids=ids, out_dist=dist, stream=s, **kw)
    for _ in range(3):
        ids.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(ids, ref[0]) and torch.equal(dist, ref[1])
    pkg.suco_free(ix)


@pytest.mark.parametrize("id_passes,cluster_size", [(2, 1), (2, 8), (4, 4), (4, 16), (8, 8), (64, 1), (16, 4)])
def test_tiny_workload_in_several_id_passes(tiny, id_passes, cluster_size):
    # the running candidate list of a multi-pass query gives the same stages
    # and results as one pass: checked against the oracle stage by stage
    w, X, Q, idx = tiny
    run(X, idx, Q[:24], w.k, w.alpha, w.beta, cluster_size=cluster_size, id_passes=id_passes)


@pytest.mark.parametrize("alpha,beta,k", [(0.01, 0.3, 10), (0.2, 0.05, 64), (1.0, 0.01, 5)])
def test_several_id_passes_with_ties_at_the_cut(tiny, alpha, beta, k):
    # small alpha with a large beta leaves many ids at score 0 (cut theta = 0,
    # ties by id across passes); alpha = 1 gives every id the score Ns
    w, X, Q, idx = tiny
    run(X, idx, Q[:12], k, alpha, beta, cluster_size=4, id_passes=8)


def test_id_passes_do_not_change_the_answer():
    X = W.random_data(11, 6000, 40, "int")
    Q = W.random_data(12, 64, 40, "int")
    idx = oracle.build_index(X, 5, 9, 3, W.random_init_ids(13, 6000, 5, 9))
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).cuda(), 5, 9, idx["centroids"], idx["assign"])
    try:
        Qd = torch.from_numpy(Q).cuda()
        ref = pkg.suco_query_batch(ix, Qd, 16, 0.1, 0.05)
        for P, CL in ((2, 2), (4, 16), (32, 2), (64, 1)):
            got = pkg.suco_query_batch(ix, Qd, 16, 0.1, 0.05, id_passes=P, cluster_size=CL)
            torch.cuda.synchronize()
            assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1]), (P, CL)
        with pytest.raises(pkg.SucoError):
            pkg.suco_query_batch(ix, Qd, 16, 0.1, 0.05, id_passes=3)
        with pytest.raises(pkg.SucoError):
            pkg.suco_query_batch(ix, Qd, 16, 0.1, 0.05, id_passes=128)
    finally:
        pkg.suco_free(ix)


@pytest.mark.parametrize("cluster_size,id_passes", [(4, 0), (8, 2)])
def test_stage_clocks_leave_the_answer_unchanged_and_are_ordered(tiny, cluster_size, id_passes):
    from paper_2411_14754_gb300 import stage_profile
    w, X, Q, idx = tiny
    Xd = torch.from_numpy(X).cuda()
    Qd = torch.from_numpy(Q).cuda()
    ix = pkg.suco_build_index_from_assignments(Xd, idx["Ns"], idx["sqrtK"], idx["centroids"], idx["assign"])
    try:
        kw = dict(cluster_size=cluster_size, id_passes=id_passes)
        ids, dist = pkg.suco_query_batch(ix, Qd, w.k, w.alpha, w.beta, **kw)
        out = pkg.suco_query_debug(ix, Qd, w.k, w.alpha, w.beta, want=("stage_clock",), **kw)
        torch.cuda.synchronize()
        assert torch.equal(out["ids"], ids) and torch.equal(out["dist"], dist)
        clk = out["stage_clock"].cpu().numpy()
    finally:
        pkg.suco_free(ix)
    assert (clk[:, cluster_size:, :] == -1).all()            # rows past the cluster are not written
    c = clk[:, :cluster_size, :]
    assert (c[:, :, 0] >= 0).all()                           # SM ids
    assert (np.diff(c[:, :, 1:16], axis=2) >= 0).all()      # stamps in stage order
    assert (c[:, 0, 16] >= c[:, 0, 15]).all() and (clk[:, 1:cluster_size, 16] == -1).all()
    assert (c[:, :, 18] > 0).all() and (c[:, :, 19] > 0).all()
    res = stage_profile.summarise(clk)
    assert res["cluster_size"] == cluster_size
    assert abs(sum(r["share"] for r in res["stages"][:-1]) - 1.0) < 1e-9
