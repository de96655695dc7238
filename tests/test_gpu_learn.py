"""Learned per-query ratios on the GPU: kernels against the FP64 network oracle,
the predict path against features + forward, learned queries against the
query oracle, and what the trained network gains over fixed ratios.

Weights are BF16 on the GPU; the oracle takes the same BF16-rounded values in
FP64, so the remaining differences are FP32 sums and erff (tolerances below
are a few hundred FP32 ulps of the largest term)."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import mlp_oracle as M
import paper_2411_14754_gb300 as pkg
from paper_2411_14754_gb300 import learn as L
from paper_2411_14754_gb300 import workloads as W
from parity_util import assert_topk_matches

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2411_14754_gb300 import build
    build.build()
    pkg.load_library()


@pytest.fixture(scope="module")
def small():
    """Workload-5 shaped data at n = 20000 with the oracle's index."""
    w = W.WORKLOADS[5]
    n, sk = 20_000, 16
    X = W.dataset(5, n=n)
    idx = oracle.build_index(X, w.Ns, sk, 4, W.random_init_ids(51, n, w.Ns, sk))
    ix = pkg.suco_build_index_from_assignments(torch.from_numpy(X).to(DEV), w.Ns, sk, idx["centroids"],
                                               idx["assign"])
    Q = W.queries(5, nq=64)
    yield w, X, idx, ix, Q
    pkg.suco_free(ix)


def _model(F, H, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    m = L.Mlp(F, H, seed=seed)
    t = m.tensors
    t["W1"].copy_(torch.from_numpy(rng.standard_normal((F, H)).astype(np.float32) * scale / math.sqrt(F)))
    t["b1"].copy_(torch.from_numpy(rng.standard_normal(H).astype(np.float32) * 0.3))
    t["W2"].copy_(torch.from_numpy(rng.standard_normal((H, 2)).astype(np.float32) / math.sqrt(H)))
    t["b2"].copy_(torch.from_numpy(rng.standard_normal(2).astype(np.float32)))
    t["mean"].copy_(torch.from_numpy(rng.standard_normal(F).astype(np.float32)))
    t["std"].copy_(torch.from_numpy((rng.random(F) + 0.5).astype(np.float32)))
    t["w1b"] = t["W1"].to(torch.bfloat16)
    t["w2b"] = t["W2"].to(torch.bfloat16)
    return m


def _oracle_params(m):
    t = m.tensors
    f64 = lambda x: x.float().cpu().numpy().astype(np.float64)  # noqa: E731
    return dict(mean=f64(t["mean"]), std=f64(t["std"]), W1=f64(t["w1b"]), b1=f64(t["b1"]), W2=f64(t["w2b"]),
                b2=f64(t["b2"]))


def _close(gpu, ref, rel=2e-5):
    gpu = np.asarray(gpu, np.float64)
    scale = max(float(np.abs(ref).max()), 1e-30)
    np.testing.assert_allclose(gpu, ref, rtol=0, atol=rel * scale)


def test_features_match_the_oracle(small):
    w, X, idx, ix, Q = small
    f = pkg.suco_query_features(ix, torch.from_numpy(Q).to(DEV)).cpu().numpy()
    Ns = w.Ns
    for b in range(16):
        o = M.features(X, idx, Q[b])
        # nearest-centroid distances: the ranking's own FP32 arithmetic, bit for bit
        np.testing.assert_array_equal(f[b, :2 * Ns].astype(np.float64), o[:2 * Ns])
        # cell sizes: exact integers through log1p
        np.testing.assert_array_equal(np.rint(np.expm1(f[b, 2 * Ns:].astype(np.float64))),
                                      np.rint(np.expm1(o[2 * Ns:])))
        np.testing.assert_allclose(f[b, 2 * Ns:], o[2 * Ns:], rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("F,H,B", [(48, 256, 300), (3, 1, 1), (7, 33, 17), (96, 512, 64)])
def test_forward_matches_the_oracle(F, H, B):
    m = _model(F, H, seed=F * 1000 + H)
    x = torch.from_numpy(np.random.default_rng(B).standard_normal((B, F)).astype(np.float32) * 3 + 1).to(DEV)
    z1 = torch.empty((B, H), device=DEV)
    h = torch.empty((B, H), device=DEV)
    y = pkg.suco_mlp_forward(m.struct(), x, z1, h)
    p = _oracle_params(m)
    ref = M.forward(x.cpu().numpy().astype(np.float64), **p)
    _close(z1.cpu().numpy(), ref["z1"])
    _close(h.cpu().numpy(), ref["h"])
    _close(y.cpu().numpy(), ref["y"])


@pytest.mark.parametrize("F,H,B", [(48, 256, 512), (5, 40, 3), (96, 512, 1)])
def test_backward_matches_the_oracle(F, H, B):
    m = _model(F, H, seed=7 + F + H)
    rng = np.random.default_rng(11 + B)
    x = torch.from_numpy(rng.standard_normal((B, F)).astype(np.float32) * 2).to(DEV)
    tg = torch.from_numpy(rng.standard_normal((B, 2)).astype(np.float32)).to(DEV)
    z1, h, dz1 = (torch.empty((B, H), device=DEV) for _ in range(3))
    dy = torch.empty((B, 2), device=DEV)
    g = {k: torch.full_like(m.tensors[k], float("nan")) for k in ("W1", "b1", "W2", "b2")}
    loss = torch.full((1,), float("nan"), device=DEV)
    st = m.struct()
    y = pkg.suco_mlp_forward(st, x, z1, h)
    pkg.suco_mlp_backward(st, x, z1, h, y, tg, dz1, dy, g["W1"], g["b1"], g["W2"], g["b2"], loss)
    p = _oracle_params(m)
    lo, go, _ = M.loss_and_grads(x.cpu().numpy().astype(np.float64), tg.cpu().numpy().astype(np.float64), **p)
    assert abs(float(loss.item()) - lo) <= 1e-5 * max(lo, 1e-30)
    for k in ("W1", "b1", "W2", "b2"):
        _close(g[k].cpu().numpy(), go[k], rel=5e-5)
    _close(dz1.cpu().numpy(), go["dz1"], rel=5e-5)
    _close(dy.cpu().numpy(), go["dy"], rel=1e-6)


def test_adamw_matches_the_oracle_over_several_steps():
    rng = np.random.default_rng(3)
    n = 1000
    p = rng.standard_normal(n)
    m = np.zeros(n)
    v = np.zeros(n)
    pd = torch.from_numpy(p.astype(np.float32)).to(DEV)
    md, vd = torch.zeros(n, device=DEV), torch.zeros(n, device=DEV)
    cp = torch.empty(n, dtype=torch.bfloat16, device=DEV)
    p = pd.cpu().numpy().astype(np.float64)
    for step in range(1, 6):
        g = rng.standard_normal(n)
        gd = torch.from_numpy(g.astype(np.float32)).to(DEV)
        g = gd.cpu().numpy().astype(np.float64)
        pkg.suco_adamw_step(pd, gd, md, vd, 1e-2, step, weight_decay=0.1, bf16_copy=cp)
        p, m, v = M.adamw(p, g, m, v, lr=1e-2, step=step, wd=0.1)
        np.testing.assert_allclose(pd.cpu().numpy(), p, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(md.cpu().numpy(), m, rtol=1e-5, atol=1e-7)
        # the BF16 copy is the round-to-nearest-even of the FP32 master
        assert torch.equal(cp, pd.to(torch.bfloat16))


def test_predict_is_features_then_forward_then_clamp(small):
    w, X, idx, ix, Q = small
    F = 3 * w.Ns
    m = _model(F, 256, seed=5, scale=0.3)
    Qd = torch.from_numpy(Q).to(DEV)
    off = (0.25, -0.5)
    alpha, beta = L.predict(ix, m, Qd, offsets=off)
    feats = pkg.suco_query_features(ix, Qd)
    y = pkg.suco_mlp_forward(m.struct(), feats).cpu().numpy().astype(np.float64)
    la = np.clip(y[:, 0] + off[0], math.log(L.ALPHA_RANGE[0]), math.log(L.ALPHA_RANGE[1]))
    lb = np.clip(y[:, 1] + off[1], math.log(L.BETA_RANGE[0]), math.log(L.BETA_RANGE[1]))
    np.testing.assert_allclose(alpha.cpu().numpy(), np.exp(la), rtol=1e-5)
    np.testing.assert_allclose(beta.cpu().numpy(), np.exp(lb), rtol=1e-5)
    # a non-finite output falls back to the fixed ratios
    m.tensors["b2"].fill_(float("nan"))
    alpha, beta = L.predict(ix, m, Qd)
    assert (alpha.cpu().numpy() == np.float32(L.FALLBACK[0])).all()
    assert (beta.cpu().numpy() == np.float32(L.FALLBACK[1])).all()


def test_learned_queries_match_the_query_oracle(small):
    w, X, idx, ix, Q = small
    m = _model(3 * w.Ns, 256, seed=9, scale=0.5)
    Qd = torch.from_numpy(Q[:24]).to(DEV)
    alpha, beta = L.predict(ix, m, Qd)
    ids, dist = L.query_learned(ix, m, Qd, w.k)
    al, be = alpha.cpu().numpy(), beta.cpu().numpy()
    assert len(set(np.round(al, 6).tolist())) > 1     # the ratios really differ per query
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
    n = X.shape[0]
    for b in range(len(al)):
        T = oracle.collision_threshold(float(al[b]), n)
        C = oracle.candidate_count(min(float(be[b]), L.BETA_RANGE[1]), n, w.k)
        o = oracle.query(X, idx, Q[b], w.k, T, C, rank_precision=1)
        assert_topk_matches(X, Q[b], ids[b], dist[b], o["ids"], o["dist"])


def test_training_step_matches_the_oracle(small):
    # one step of the GPU recipe (forward, backward, AdamW on every tensor)
    # against the same step in FP64
    w, X, idx, ix, Q = small
    F, H, B = 3 * w.Ns, 64, 128
    m = _model(F, H, seed=13)
    rng = np.random.default_rng(17)
    x = torch.from_numpy(rng.standard_normal((B, F)).astype(np.float32)).to(DEV)
    tg = torch.from_numpy(rng.standard_normal((B, 2)).astype(np.float32)).to(DEV)
    p0 = {k: m.tensors[k].cpu().numpy().astype(np.float64) for k in ("W1", "b1", "W2", "b2")}
    po = _oracle_params(m)
    _, go, _ = M.loss_and_grads(x.cpu().numpy().astype(np.float64), tg.cpu().numpy().astype(np.float64), **po)
    L.train(m, x, tg, epochs=1, batch=B, lr=1e-3, weight_decay=1e-4)
    for k in ("W1", "b1", "W2", "b2"):
        pk, _, _ = M.adamw(p0[k], go[k], np.zeros_like(p0[k]), np.zeros_like(p0[k]), lr=1e-3, step=1,
                           wd=1e-4 if k in ("W1", "W2") else 0.0)
        # the first AdamW step is lr * sign(g) (+ decay) except where |g| is tiny
        big = np.abs(go[k]) > 1e-3 * np.abs(go[k]).max()
        np.testing.assert_allclose(m.tensors[k].cpu().numpy()[big], pk[big], rtol=1e-5, atol=1e-6)


def test_training_fits_a_smooth_target():
    rng = np.random.default_rng(23)
    F, N = 12, 8192
    x = rng.standard_normal((N, F)).astype(np.float32)
    A = rng.standard_normal((F, 2)) * 0.5
    t = (np.tanh(x @ A) + 0.1 * x[:, :2] ** 2).astype(np.float32)
    xd, td = torch.from_numpy(x).to(DEV), torch.from_numpy(t).to(DEV)
    m = L.Mlp(F, 128, seed=1)
    m.set_standardisation(xd)
    m.set_output_bias(td)
    hist = L.train(m, xd, td, epochs=40, batch=512, lr=3e-3)
    base = float(((t - t.mean(0)) ** 2).sum() / (2 * N))    # loss of the best constant
    assert hist[-1] < 0.1 * base, (hist, base)
    assert hist[-1] < hist[0]


def test_trained_network_beats_fixed_ratios_at_the_same_recall():
    """The recipe on a workload-5 shaped index (n = 100000): training queries
    give grid labels, the network is trained on the GPU, its margin is tuned on
    a validation split, and on held-out queries it must reach the target mean
    recall@10 (judged against the FP64 oracle's exact k-NN) while moving fewer
    bytes on average than the cheapest fixed grid point that reaches it."""
    w = W.WORKLOADS[5]
    n, sk, k, target = 100_000, 32, 10, 0.95
    X = W.dataset(5, n=n)
    Xd = torch.from_numpy(X).to(DEV)
    ix = pkg.suco_build_index(Xd, w.Ns, sk, 10, init_ids=W.random_init_ids(52, n, w.Ns, sk))
    try:
        Qt = torch.from_numpy(W.queries(5, nq=12_000, train=True)).to(DEV)
        model, rep = L.fit(ix, Xd, Qt, k, epochs=40, target=target)
        Qh = W.queries(5, nq=600)
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(oracle.max_threads()) as ex:
            gt = np.stack(list(ex.map(lambda q: oracle.bruteforce_knn(X, q, k)[0], Qh)))
        Qhd = torch.from_numpy(Qh).to(DEV)
        ids, _ = L.query_learned(ix, model, Qhd, k)
        r_learned = float(L.recall_rows(ids.cpu().numpy(), gt).mean())
        alpha, beta = L.predict(ix, model, Qhd)
        a = alpha.cpu().numpy().astype(np.float64)
        b = beta.cpu().numpy().astype(np.float64)
        learned_bytes = float(np.mean(L.path_bytes(a, b, n, X.shape[1], w.Ns)))
        rec = L.grid_recalls(ix, Qhd, gt, k).mean(axis=0)
        fa, fb = L.cheapest_fixed(rec, n, X.shape[1], w.Ns, target=target)
        fixed_bytes = L.path_bytes(fa, fb, n, X.shape[1], w.Ns)
        print(dict(rep, held_out_recall=r_learned, learned_bytes=learned_bytes, fixed=(fa, fb),
                   fixed_recall=float(rec[L.ALPHA_GRID.index(fa), L.BETA_GRID.index(fb)]), fixed_bytes=fixed_bytes))
        assert rep["loss_last"] < rep["loss_first"]
        assert r_learned >= target - 0.01
        assert learned_bytes < fixed_bytes
    finally:
        pkg.suco_free(ix)
