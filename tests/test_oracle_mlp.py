"""Pins of the FP64 oracle of the learned-ratio network (CPU only)."""
import math

import numpy as np
from scipy.spatial.distance import cdist
from scipy.stats import norm

import oracle
from oracle import mlp_oracle as M
from paper_2411_14754_gb300 import workloads as W


def test_gelu_closed_forms():
    assert M.gelu(0.0) == 0.0
    assert abs(M.gelu_grad(0.0) - 0.5) < 1e-15
    np.testing.assert_allclose(M.gelu(1.0), norm.cdf(1.0), rtol=1e-14)           # z * Phi(z) at z = 1
    np.testing.assert_allclose(M.gelu(-2.0), -2.0 * norm.cdf(-2.0), rtol=1e-14)
    assert abs(M.gelu(12.0) - 12.0) < 1e-12 and abs(M.gelu(-12.0)) < 1e-12
    # derivative against a central difference of the function itself
    for z in (-3.0, -0.7, 0.3, 2.5):
        fd = (M.gelu(z + 1e-6) - M.gelu(z - 1e-6)) / 2e-6
        assert abs(fd - M.gelu_grad(z)) < 1e-8


def _net(seed, F=6, H=7, B=5):
    rng = np.random.default_rng(seed)
    return dict(x=rng.standard_normal((B, F)), t=rng.standard_normal((B, 2)), mean=rng.standard_normal(F),
                std=rng.random(F) + 0.5, W1=rng.standard_normal((F, H)), b1=rng.standard_normal(H),
                W2=rng.standard_normal((H, 2)), b2=rng.standard_normal(2))


def test_gradients_match_central_differences():
    for seed in range(4):
        n = _net(seed)
        loss, g, _ = M.loss_and_grads(n["x"], n["t"], n["mean"], n["std"], n["W1"], n["b1"], n["W2"], n["b2"])
        for name in ("W1", "b1", "W2", "b2"):
            p = n[name]
            it = np.nditer(p, flags=["multi_index"])
            for _ in it:
                ix = it.multi_index
                old = p[ix]
                p[ix] = old + 1e-6
                lp, _, _ = M.loss_and_grads(n["x"], n["t"], n["mean"], n["std"], n["W1"], n["b1"], n["W2"], n["b2"])
                p[ix] = old - 1e-6
                lm, _, _ = M.loss_and_grads(n["x"], n["t"], n["mean"], n["std"], n["W1"], n["b1"], n["W2"], n["b2"])
                p[ix] = old
                fd = (lp - lm) / 2e-6
                assert abs(fd - g[name][ix]) <= 1e-6 * max(1.0, abs(fd)), (name, ix, fd, g[name][ix])


def test_zero_output_layer_gives_bias_and_no_hidden_gradient():
    n = _net(9)
    W2 = np.zeros_like(n["W2"])
    f = M.forward(n["x"], n["mean"], n["std"], n["W1"], n["b1"], W2, n["b2"])
    np.testing.assert_array_equal(f["y"], np.tile(n["b2"], (n["x"].shape[0], 1)))
    _, g, _ = M.loss_and_grads(n["x"], n["t"], n["mean"], n["std"], n["W1"], n["b1"], W2, n["b2"])
    assert not g["W1"].any() and not g["b1"].any()
    # with zero output weights the bias gradient is the mean residual
    np.testing.assert_allclose(g["b2"], (n["b2"] - n["t"]).sum(axis=0) / n["x"].shape[0], rtol=1e-12)


def test_adamw_first_step_is_a_signed_lr_step():
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = M.adamw(np.ones(3), g, np.zeros(3), np.zeros(3), lr=0.01, step=1, eps=0.0)
    np.testing.assert_allclose(p, 1.0 - 0.01 * np.sign(g), rtol=1e-12)
    p2, _, _ = M.adamw(np.ones(3), np.zeros(3), np.zeros(3), np.zeros(3), lr=0.01, step=1, wd=0.5)
    np.testing.assert_allclose(p2, 1.0 - 0.01 * 0.5, rtol=1e-12)      # decoupled decay only


def test_features_from_a_direct_computation():
    X = W.dataset(1, n=2000)
    idx = oracle.build_index(X, 8, 6, 2, W.random_init_ids(3, 2000, 8, 6))
    q = W.queries(1, nq=1)[0]
    f = M.features(X, idx, q)
    for i in range(8):
        cells = []
        for h in range(2):
            off, ln = oracle.half_dims(128, 8, i, h)
            c = idx["centroids"][i, h, :, :ln].astype(np.float64)
            dd = cdist(q[None, off:off + ln].astype(np.float64), c, "sqeuclidean")[0]
            a = int(np.argmin(dd))
            cells.append(a)
            np.testing.assert_allclose(f[2 * i + h], dd[a], rtol=1e-6)     # FP32 ranking distances vs FP64
        size = int(((idx["assign"][i, 0] == cells[0]) & (idx["assign"][i, 1] == cells[1])).sum())
        assert abs(f[16 + i] - math.log1p(size)) < 1e-12
