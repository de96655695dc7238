"""Pins of the reduced-precision oracle (oracle/precision_oracle.py) against
the number formats' definitions, library conversions and closed forms."""
import numpy as np
import pytest

import oracle
from oracle import precision_oracle as P

torch = pytest.importorskip("torch")


def test_bf16_rounding_matches_torch_round_to_nearest_even():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(50_000) * 1e3, rng.standard_normal(50_000) * 1e-30,
                        [0.0, -0.0, 1.0, 255.0, 3.4e38, -3.4e38, np.inf, -np.inf]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(P.round_bf16(x), ref)


def test_bf16_ties_go_to_even():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: rounds down to the even 1.0;
    # 1 + 3*2^-8 lies halfway between 1 + 2^-7 and 1 + 2^-6: rounds up to the even one
    x = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8], dtype=np.float32)
    np.testing.assert_array_equal(P.bf16_to_f64(P.round_bf16(x)), [1.0, 1 + 2.0 ** -6])


def test_bf16_is_exact_on_small_integers():
    x = np.arange(0, 257, dtype=np.float32)
    np.testing.assert_array_equal(P.bf16_to_f64(P.round_bf16(x)), x.astype(np.float64))


def test_e4m3_table_closed_form():
    v = P.e4m3_values()
    assert np.nanmax(v) == 448.0 and np.nanmin(v) == -448.0
    assert v[0x01] == 2.0 ** -9          # smallest subnormal
    assert v[0x08] == 2.0 ** -6          # smallest normal
    assert v[0x38] == 1.0
    assert np.isnan(v[0x7F]) and np.isnan(v[0xFF])
    assert np.isfinite(v).sum() == 254


def test_e4m3_quantisation_matches_torch_cast():
    rng = np.random.default_rng(1)
    v = P.e4m3_values()
    fin = v[np.isfinite(v)]
    mids = ((np.sort(fin)[1:] + np.sort(fin)[:-1]) / 2.0)  # every tie point
    x = np.concatenate([rng.uniform(-440, 440, 3000), rng.uniform(-1, 1, 2000) * 2.0 ** -5, mids]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    got = P.quantize_e4m3(x.astype(np.float64))
    # +0 / -0 are both exact for a zero tie; compare values
    np.testing.assert_array_equal(P.e4m3_to_f64(got), P.e4m3_to_f64(ref))


def test_e4m3_saturates():
    np.testing.assert_array_equal(P.e4m3_to_f64(P.quantize_e4m3(np.array([1e6, -1e6, 449.0]))), [448.0, -448.0, 448.0])


def test_coarse_rerank_with_all_survivors_is_the_exact_rerank():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((500, 24)).astype(np.float32)
    q = rng.standard_normal(24).astype(np.float32)
    cands = rng.choice(500, 120, replace=False)
    Xh = P.decoded_rows(X[cands], 1)
    out = P.coarse_rerank(X, Xh, q, cands, R=10_000, k=7)
    ids, dist = oracle.rerank(X, q, cands, 7)
    assert np.array_equal(out["ids"], ids)
    np.testing.assert_array_equal(out["dist"], dist)


def test_coarse_rerank_on_exactly_representable_data_keeps_the_true_nearest():
    # integer rows <= 256 are exact in BF16: coarse = exact distance, so the
    # R survivors are the R nearest candidates and the top-k is the exact top-k
    rng = np.random.default_rng(3)
    X = rng.integers(0, 256, size=(800, 16)).astype(np.float32)
    q = rng.integers(0, 256, size=16).astype(np.float32)
    cands = np.arange(800)
    out = P.coarse_rerank(X, P.decoded_rows(X, 1), q, cands, R=20, k=5)
    exact = ((X.astype(np.float64) - q) ** 2).sum(1)
    order = np.lexsort((cands, exact))
    assert np.array_equal(np.sort(out["survivors"]), np.sort(cands[order[:20]]))
    assert np.array_equal(out["ids"], cands[order[:5]])


def test_e4m3_rows_use_one_scale_per_subspace():
    rng = np.random.default_rng(4)
    X = np.abs(rng.standard_normal((300, 12))).astype(np.float32)
    X[:, 8:] *= 1000.0  # subspace 2 of 3 has a much larger range
    s = P.subspace_scales_e4m3(X, 3)
    assert s[2] == pytest.approx(np.abs(X[:, 8:]).max() / 448.0)
    Xh = P.decoded_rows(X, 2, Ns=3, scales=s)
    # relative error of a normal E4M3 value is at most 2^-4
    big = np.abs(X) > 2.0 ** -6 * np.repeat(s, 4)[None, :]
    rel = np.abs(Xh - X)[big] / np.abs(X)[big]
    assert rel.max() <= 2.0 ** -4 + 1e-12


def test_bf16_centroid_tables_on_bf16_exact_data_are_the_fp64_distances():
    # integers in [0, 16) and centroids that are data rows (no Lloyd update)
    # are exact in BF16: the tables are then the FP64 squared distances of the
    # raw half-vectors, and the norms |q_h|^2 + |c|^2 by direct sums
    from scipy.spatial.distance import cdist
    from paper_2411_14754_gb300 import workloads as W
    n, d, Ns, sk = 1500, 20, 2, 7
    X = W.random_data(41, n, d, kind="int")
    idx = oracle.build_index(X, Ns, sk, 0, W.random_init_ids(42, n, Ns, sk))
    for q in W.random_data(43, 4, d, kind="int"):
        tab, norms = P.bf16_centroid_tables(idx, q)
        for i in range(Ns):
            for h in range(2):
                off, ln = oracle.half_dims(d, Ns, i, h)
                c = idx["centroids"][i, h, :, :ln].astype(np.float64)
                qh = q[off:off + ln].astype(np.float64)
                np.testing.assert_array_equal(tab[i, h], cdist(qh[None, :], c, "sqeuclidean")[0])
                np.testing.assert_array_equal(norms[i, h], np.dot(qh, qh) + np.einsum("ij,ij->i", c, c))


def test_bf16_centroid_tables_round_both_operands_like_torch():
    # on general data the tables are the distances of the BF16-rounded vectors
    # (rounding by torch's bfloat16 cast, a library conversion)
    from paper_2411_14754_gb300 import workloads as W
    n, d, Ns, sk = 1200, 24, 3, 6
    X = W.random_data(44, n, d, kind="gauss") * 7.3
    idx = oracle.build_index(X, Ns, sk, 2, W.random_init_ids(45, n, Ns, sk))
    q = W.random_data(46, 1, d, kind="gauss")[0] * 7.3
    tab, _ = P.bf16_centroid_tables(idx, q)
    qb = torch.from_numpy(q).to(torch.bfloat16).double().numpy()
    for i in range(Ns):
        for h in range(2):
            off, ln = oracle.half_dims(d, Ns, i, h)
            cb = torch.from_numpy(np.ascontiguousarray(idx["centroids"][i, h, :, :ln])).to(torch.bfloat16).double()
            ref = ((cb.numpy() - qb[off:off + ln][None, :]) ** 2).sum(axis=1)
            np.testing.assert_allclose(tab[i, h], ref, rtol=1e-14, atol=0)


def test_fp8_centroid_tables_on_e4m3_exact_data_are_the_fp64_distances():
    # data whose every value is a small integer times 2^-3, a scale that
    # divides exactly: with the data scale and the query scale chosen so that
    # every quotient is an E4M3 value, the codes are exact and the tables are
    # the FP64 squared distances of the raw half-vectors
    from scipy.spatial.distance import cdist
    from paper_2411_14754_gb300 import workloads as W
    n, d, Ns, sk = 1200, 16, 2, 5
    rng = np.random.default_rng(47)
    X = (rng.integers(0, 8, size=(n, d)) * 0.125).astype(np.float32)
    X[0, :] = 0.875                                # max|x| = 7/8 in every subspace
    idx = oracle.build_index(X, Ns, sk, 0, W.random_init_ids(48, n, Ns, sk))
    s = P.subspace_scales_e4m3(X, Ns)              # (7/8) / 448 = 2^-9: quotients x * 2^9 are exact
    assert (s == np.float32(2.0 ** -9)).all()
    for q in (rng.integers(0, 8, size=(3, d)) * 0.125).astype(np.float32):
        q[[0, 8]] = 0.875                          # the query's scale is 2^-9 too
        tab, norms = P.fp8_centroid_tables(idx, q, s)
        for i in range(Ns):
            for h in range(2):
                off, ln = oracle.half_dims(d, Ns, i, h)
                c = idx["centroids"][i, h, :, :ln].astype(np.float64)
                qh = q[off:off + ln].astype(np.float64)
                np.testing.assert_array_equal(tab[i, h], cdist(qh[None, :], c, "sqeuclidean")[0])
                np.testing.assert_array_equal(norms[i, h], np.dot(qh, qh) + np.einsum("ij,ij->i", c, c))


def test_fp8_centroid_tables_code_both_operands_like_torch():
    # general data: values are torch's float8_e4m3fn casts of the FP32
    # quotients (a library conversion; no saturation is reached here) times the scales
    from paper_2411_14754_gb300 import workloads as W
    n, d, Ns, sk = 1500, 30, 3, 6
    X = np.abs(W.random_data(49, n, d, kind="gauss")) * np.float32(5.0)
    idx = oracle.build_index(X, Ns, sk, 2, W.random_init_ids(50, n, Ns, sk))
    s = P.subspace_scales_e4m3(X, Ns)
    q = np.abs(W.random_data(51, 1, d, kind="gauss")[0]) * np.float32(5.0)
    tab, _ = P.fp8_centroid_tables(idx, q, s)

    def coded(v, scale):
        quot = torch.from_numpy(np.ascontiguousarray(v / np.float32(scale), dtype=np.float32))
        return quot.to(torch.float8_e4m3fn).double().numpy() * float(scale)

    for i in range(Ns):
        so, sl = oracle.subspace_dims(d, Ns, i)
        t = np.float32(np.abs(q[so:so + sl]).max() / np.float32(448.0))
        for h in range(2):
            off, ln = oracle.half_dims(d, Ns, i, h)
            qc = coded(q[off:off + ln], t)
            cc = coded(idx["centroids"][i, h, :, :ln], s[i])
            np.testing.assert_allclose(tab[i, h], ((cc - qc[None, :]) ** 2).sum(1), rtol=1e-14, atol=0)
