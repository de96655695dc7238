"""Comparison helpers shared by the GPU parity tests (test-side only)."""
import numpy as np

import oracle
from oracle import precision_oracle as P

# FP32 re-rank distances against the FP64 oracle (tolerance of the FP32 path)
RTOL = 1e-5
# FP32 sum of d non-negative terms vs FP64, relative, at the R-th coarse distance
COARSE_RTOL = 2e-5


def true_sqdist(X, q, ids):
    ids = np.asarray(ids)
    ok = ids >= 0
    out = np.full(len(ids), np.inf)
    diff = X[ids[ok]].astype(np.float64) - q.astype(np.float64)[None, :]
    out[ok] = (diff * diff).sum(axis=1)
    return out


def assert_topk_matches(X, q, gpu_ids, gpu_dist, o_ids, o_dist, rtol=RTOL):
    """GPU top-k vs the oracle's: same distances within rtol at every rank; the
    id sets may differ only by ids whose distance ties the k-th one within rtol;
    every returned distance is the true distance of its id within rtol."""
    gpu_ids = np.asarray(gpu_ids, dtype=np.int64)
    gpu_dist = np.asarray(gpu_dist, dtype=np.float64)
    o_ids = np.asarray(o_ids, dtype=np.int64)
    pad_g, pad_o = gpu_ids < 0, o_ids < 0
    assert (pad_g == pad_o).all(), (gpu_ids, o_ids)
    assert np.isinf(gpu_dist[pad_g]).all()
    real = ~pad_g
    if not real.any():
        return
    td = true_sqdist(X, q, gpu_ids[real])
    np.testing.assert_allclose(gpu_dist[real], td, rtol=rtol, atol=1e-30)
    assert (np.diff(gpu_dist[real]) >= 0).all()
    np.testing.assert_allclose(gpu_dist[real], o_dist[real], rtol=rtol, atol=1e-30)
    sg, so = set(gpu_ids[real].tolist()), set(o_ids[real].tolist())
    dk = float(o_dist[real][-1])
    for i in sg ^ so:
        di = true_sqdist(X, q, [i])[0]
        assert abs(di - dk) <= rtol * max(dk, 1e-30) * 2, (i, di, dk)


def check_query_against_oracle(X, idx_o, q, gpu, b, k, T, C, stages=True):
    """Compare one query's GPU outputs (dict of host arrays, row b) with the oracle
    run in the kernel's FP32 ranking precision."""
    o = oracle.query(X, idx_o, q, k, T, C, rank_precision=1, debug=True)
    if stages:
        if "dtab" in gpu:
            np.testing.assert_array_equal(gpu["dtab"][b].astype(np.float64), o["dtab"])
        if "t_eff" in gpu:
            np.testing.assert_array_equal(gpu["t_eff"][b], o["teff"])
        if "activated" in gpu:
            np.testing.assert_array_equal(gpu["activated"][b], o["activated"])
        if "scores" in gpu:
            np.testing.assert_array_equal(gpu["scores"][b].astype(np.int32), o["scores"])
        if "cands" in gpu:
            gc = gpu["cands"][b].astype(np.int64)
            assert len(gc) == C
            assert sorted(gc.tolist()) == sorted(o["cands"].tolist())
    assert_topk_matches(X, q, gpu["ids"][b], gpu["dist"][b], o["ids"], o["dist"])
    return o


def check_coarse_against_oracle(X, q, gpu_cands, gpu_surv, gpu_ids, gpu_dist, o_cands, k, R, prec, Ns=None,
                                scales=None):
    """One query of the BF16/FP8 coarse re-rank vs the reduced-precision oracle.
    gpu_cands: the GPU's candidate ids; gpu_surv: ids flagged as survivors;
    o_cands: the oracle's candidates (same set).  The survivors must be the R
    candidates with the smallest (coarse distance, id), up to candidates whose
    coarse distance ties the R-th within FP32 rounding; the result must be the
    exact top-k of the GPU's own survivors.  Returns the oracle's coarse pass."""
    cands = np.asarray(o_cands, dtype=np.int64)
    C = len(cands)
    assert sorted(np.asarray(gpu_cands).tolist()) == sorted(cands.tolist())
    rows = P.decoded_rows(X[cands], 1) if prec == "bf16" else P.decoded_rows(X[cands], 2, Ns, scales)
    ref = P.coarse_rerank(X, rows, q, cands, R, k)
    g_surv = np.asarray(gpu_surv, dtype=np.int64)
    if C > R:
        assert len(g_surv) == R
        coarse = dict(zip(cands.tolist(), ref["coarse"].tolist()))
        cR = np.sort(ref["coarse"])[R - 1]
        for i in set(g_surv.tolist()) ^ set(ref["survivors"].tolist()):
            assert abs(coarse[i] - cR) <= COARSE_RTOL * max(cR, 1e-30), (i, coarse[i], cR)
        ids_s, dist_s = oracle.rerank(X, q, g_surv, k)
    else:
        ids_s, dist_s = oracle.rerank(X, q, cands, k)
    assert_topk_matches(X, q, gpu_ids, gpu_dist, ids_s, dist_s)
    return ref
