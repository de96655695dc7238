"""Parity at full size, in the launch configurations the benchmark times:
1,000,000 SIFT-like points (d=128, Ns=8, sqrtK=50, k=50), 1,000,000 points of
the hard mixture (d=256, Ns=16, sqrtK=50, k=10; per-query alpha and beta from
the ratio network) and 1,000,000 GIST-like points (d=960, Ns=16, sqrtK=64,
k=10; FP32, BF16 and FP8 re-rank), one batch of 1024 queries each.

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
from parity_util import assert_topk_matches, check_coarse_against_oracle, check_query_against_oracle, true_sqdist

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


# ---------------------------------------------------------------------------
# The benchmark's headline shape: 1,000,000 points from the hard mixture
# (d=256), Ns=16, sqrtK=50, k=10, a 1024-query launch in the automatic shape,
# with per-query alpha and beta produced by the ratio network's predict launch.

def _host(d):
    return {kk: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for kk, v in d.items()}


@pytest.fixture(scope="module")
def hard():
    from paper_2411_14754_gb300 import build
    build.build()
    w = W.WORKLOADS[5]
    X = W.dataset(5)
    Q = W.queries(5, nq=w.batch)
    idx = oracle.build_index(X, w.Ns, w.sqrtK, 1, W.kmeans_init_ids(5, w.n, w.Ns, w.sqrtK))
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).cuda(), w.Ns, w.sqrtK, idx["centroids"],
                                               idx["assign"])
    yield w, X, Q, idx, ix
    pkg.suco_free(ix)


def _per_query_thresholds(n, k, alpha, beta, beta_bound):
    """T_b and C_b as the kernel derives them from FP32 per-query ratios."""
    T = [oracle.collision_threshold(float(a), n) for a in alpha]
    C = [oracle.candidate_count(min(float(b), beta_bound), n, k) for b in beta]
    return T, C


def test_headline_shape_with_predicted_ratios_sampled_stage_parity(hard):
    from paper_2411_14754_gb300 import learn as L
    w, X, Q, idx, ix = hard
    Qd = torch.from_numpy(Q).cuda()
    # an untrained network (seeded weights, standardised on this batch) spreads
    # the ratios over the whole clamp range; the kernel takes them as given
    model = L.Mlp(3 * w.Ns, 256, seed=3)
    model.set_standardisation(pkg.suco_query_features(ix, Qd))
    al, be = L.predict(ix, model, Qd, offsets=(0.3, 0.6))
    beta_bound = L.BETA_RANGE[1]
    ids, dist = pkg.suco_query_batch(ix, Qd, w.k, L.FALLBACK[0], beta_bound, alpha_per_query=al,
                                     beta_per_query=be)      # the benchmark's launch
    torch.cuda.synchronize()
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
    a_np, b_np = al.cpu().numpy(), be.cpu().numpy()
    assert a_np.std() > 0 and b_np.std() > 0
    sample = [0, 211, 517, 888, 1023]
    sel = torch.tensor(sample, device="cuda")
    dbg = _host(pkg.suco_query_debug(ix, Qd[sel], w.k, L.FALLBACK[0], beta_bound,
                                     alpha_per_query=al[sel].contiguous(), beta_per_query=be[sel].contiguous()))
    torch.cuda.synchronize()
    Ts, Cs = _per_query_thresholds(w.n, w.k, a_np[sample], b_np[sample], beta_bound)
    for j, b in enumerate(sample):
        T, C = Ts[j], Cs[j]
        o = oracle.query(X, idx, Q[b], w.k, T, C, rank_precision=1, debug=True)
        np.testing.assert_array_equal(dbg["dtab"][j].astype(np.float64), o["dtab"])
        np.testing.assert_array_equal(dbg["t_eff"][j], o["teff"])
        np.testing.assert_array_equal(dbg["activated"][j], o["activated"])
        np.testing.assert_array_equal(dbg["scores"][j].astype(np.int32), o["scores"])
        gc = dbg["cands"][j].astype(np.int64)
        assert (gc[:C] >= 0).all() and (gc[C:] == -1).all()
        assert sorted(gc[:C].tolist()) == sorted(o["cands"].tolist())
        assert_topk_matches(X, Q[b], dbg["ids"][j], dbg["dist"][j], o["ids"], o["dist"])
        assert ids[b].tolist() == dbg["ids"][j].tolist()
        np.testing.assert_array_equal(dist[b], dbg["dist"][j])


def test_headline_shape_fixed_ratios_sampled_stage_parity(hard):
    w, X, Q, idx, ix = hard
    Qd = torch.from_numpy(Q).cuda()
    ids, dist = pkg.suco_query_batch(ix, Qd, w.k, w.alpha, w.beta)
    torch.cuda.synchronize()
    sample = [3, 640, 1000]
    dbg = _host(pkg.suco_query_debug(ix, Qd[sample], w.k, w.alpha, w.beta))
    for j, b in enumerate(sample):
        check_query_against_oracle(X, idx, Q[b], dbg, j, w.k, dbg["T"], dbg["C"])
        assert ids[b].cpu().tolist() == dbg["ids"][j].tolist()


def _fp64_activated(idx, q, T, cell_off):
    """Algorithm 3 in FP64 for every subspace of one query: the half-subspace
    tables written from the definition, the oracle's Dynamic Activation."""
    Ns, sk = idx["Ns"], idx["sqrtK"]
    d = len(q)
    out = []
    for i in range(Ns):
        tabs = []
        for h in range(2):
            off, ln = oracle.half_dims(d, Ns, i, h)
            c = idx["centroids"][i, h, :, :ln].astype(np.float64)
            tabs.append(((c - q[off:off + ln].astype(np.float64)[None, :]) ** 2).sum(1))
        sizes = np.diff(cell_off[i]).astype(np.int64)
        cells, _ = oracle.dynamic_activation(T, tabs[0], tabs[1], sizes, precision=0)
        out.append((set(cells.tolist()), tabs))
    return out


@pytest.mark.parametrize("number", [2, 5])
def test_activated_sets_against_fp64_end_to_end(number, full, hard):
    """Fraction of (query, subspace) pairs whose retrieved cells differ between
    the GPU (FP32 ranking) and the FP64 oracle, over a whole 1024-query launch.
    A difference is allowed only among cells whose FP64 sums lie within FP32
    rounding of the FP64 cut: every cell in the symmetric difference must."""
    w, X, Q, idx, ix = full if number == 2 else hard
    Qd = torch.from_numpy(Q).cuda()
    dbg = pkg.suco_query_debug(ix, Qd, w.k, w.alpha, w.beta, want=("activated",))
    torch.cuda.synchronize()
    act = dbg["activated"].cpu().numpy()
    T = dbg["T"]
    sk = w.sqrtK
    differ = 0
    for b in range(len(Q)):
        for i, (cells64, (d1, d2)) in enumerate(_fp64_activated(idx, Q[b], T, idx["cell_off"])):
            g = set(np.flatnonzero(act[b, i]).tolist())
            if g == cells64:
                continue
            differ += 1
            kappa = max(d1[c // sk] + d2[c % sk] for c in cells64)
            for c in g ^ cells64:
                s = d1[c // sk] + d2[c % sk]
                assert abs(s - kappa) <= 1e-5 * kappa, (b, i, c, s, kappa)
    frac = differ / (len(Q) * w.Ns)
    print(f"\nworkload {number}: activated sets differing from FP64 in {differ} of {len(Q) * w.Ns} "
          f"(query, subspace) pairs ({frac:.2e})")
    assert frac < 0.01


# ---------------------------------------------------------------------------
# The precision workload: 1,000,000 GIST-like points (d=960), Ns=16, sqrtK=64,
# alpha=0.03, beta=0.005 (C=5000), k=10, exact re-rank of the top R=512.

@pytest.fixture(scope="module")
def gist():
    from paper_2411_14754_gb300 import build
    from oracle import precision_oracle as P
    build.build()
    w = W.WORKLOADS[3]
    X = W.dataset(3)
    Q = W.queries(3, nq=w.batch)
    idx = oracle.build_index(X, w.Ns, w.sqrtK, 1, W.kmeans_init_ids(3, w.n, w.Ns, w.sqrtK))
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).cuda(), w.Ns, w.sqrtK, idx["centroids"],
                                               idx["assign"])
    pkg.suco_add_reduced_copies(ix, rank_bf16=False)
    scales = P.subspace_scales_e4m3(X, w.Ns)
    sample = [0, 333, 1023]
    Ts, Cs = oracle.collision_threshold(w.alpha, w.n), oracle.candidate_count(w.beta, w.n, w.k)
    ref = {b: oracle.query(X, idx, Q[b], w.k, Ts, Cs, rank_precision=1, debug=True) for b in sample}
    yield w, X, Q, idx, ix, scales, sample, ref
    pkg.suco_free(ix)


def test_precision_workload_fp32_sampled_stage_parity(gist):
    w, X, Q, idx, ix, scales, sample, ref = gist
    Qd = torch.from_numpy(Q).cuda()
    ids, dist = pkg.suco_query_batch(ix, Qd, w.k, w.alpha, w.beta)
    torch.cuda.synchronize()
    dbg = _host(pkg.suco_query_debug(ix, Qd[sample], w.k, w.alpha, w.beta))
    assert (dbg["T"], dbg["C"]) == (30_000, 5_000)
    for j, b in enumerate(sample):
        o = ref[b]
        np.testing.assert_array_equal(dbg["dtab"][j].astype(np.float64), o["dtab"])
        np.testing.assert_array_equal(dbg["t_eff"][j], o["teff"])
        np.testing.assert_array_equal(dbg["activated"][j], o["activated"])
        np.testing.assert_array_equal(dbg["scores"][j].astype(np.int32), o["scores"])
        assert sorted(dbg["cands"][j].tolist()) == sorted(o["cands"].tolist())
        assert_topk_matches(X, Q[b], dbg["ids"][j], dbg["dist"][j], o["ids"], o["dist"])
        assert ids[b].cpu().tolist() == dbg["ids"][j].tolist()


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_precision_workload_coarse_rerank_against_the_oracle(gist, prec):
    w, X, Q, idx, ix, scales, sample, ref = gist
    Qd = torch.from_numpy(Q).cuda()
    R = 512
    ids, dist = pkg.suco_query_batch(ix, Qd, w.k, w.alpha, w.beta, precision=prec, exact_rerank=R)
    torch.cuda.synchronize()
    dbg = _host(pkg.suco_query_debug(ix, Qd[sample], w.k, w.alpha, w.beta, want=("cands", "survivors"),
                                     precision=prec, exact_rerank=R))
    for j, b in enumerate(sample):
        check_coarse_against_oracle(X, Q[b], dbg["cands"][j], np.flatnonzero(dbg["survivors"][j]), dbg["ids"][j],
                                    dbg["dist"][j], ref[b]["cands"], w.k, R, prec, w.Ns, scales)
        assert ids[b].cpu().tolist() == dbg["ids"][j].tolist()
