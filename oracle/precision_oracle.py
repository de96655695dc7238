"""Reduced-precision copies of the dataset and the coarse re-rank (TEST INFRASTRUCTURE).

The paper computes in full precision.  The query path also offers a
reduced-precision re-rank: candidate rows are read from a BF16 (or FP8 E4M3,
with one scale per subspace) copy of the dataset, the R candidates with the
smallest coarse squared distance survive, and those are re-ranked exactly.
This module restates that computation in FP64 with NumPy, from the number
formats' definitions:

  - bfloat16: the upper 16 bits of an IEEE binary32 value after rounding to
    nearest, ties to even, on the dropped 16 bits (8 significant bits);
  - E4M3 (the "fn" variant): 1 sign bit, 4 exponent bits with bias 7, 3
    mantissa bits; exponent 0 encodes subnormals m/8 * 2^-6; the code with
    all exponent and mantissa bits set is NaN; there is no infinity and the
    largest finite magnitude is 448.  Rounding is to nearest, ties to even,
    and magnitudes beyond 448 saturate to 448.

Coarse distance of a candidate row x to the query q: sum_j (xhat_j - q_j)^2,
xhat the decoded reduced-precision row (times the subspace scale for E4M3).
Survivors: the first min(R, C) candidates by (coarse distance, id).  Result:
the k survivors nearest by exact squared distance, ties by id.
"""
import numpy as np

from . import suco_oracle as _o


def round_bf16(x):
    """FP32 -> bfloat16 bit patterns (uint16), round to nearest even."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    nan = np.isnan(np.asarray(x, dtype=np.float32))
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF
    r = np.where(nan, (u >> 16) | 0x40, r)  # keep NaN a (quiet) NaN
    return r.astype(np.uint16)


def bf16_to_f64(b):
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)


def e4m3_values():
    """Value of each of the 256 E4M3 codes (NaN for the two NaN codes)."""
    v = np.empty(256, dtype=np.float64)
    for c in range(256):
        s = -1.0 if c & 0x80 else 1.0
        e = (c >> 3) & 0xF
        m = c & 0x7
        if e == 0xF and m == 0x7:
            v[c] = np.nan
        elif e == 0:
            v[c] = s * (m / 8.0) * 2.0 ** -6
        else:
            v[c] = s * (1.0 + m / 8.0) * 2.0 ** (e - 7)
    return v


def quantize_e4m3(x):
    """float -> E4M3 codes (uint8): nearest finite value, ties to the even
    code (mantissa LSB 0), magnitudes beyond 448 saturated, the sign bit of a
    negative input kept.  The non-negative codes 0x00..0x7E have increasing
    values, so the magnitude's two neighbours are found by a sorted search."""
    pos = e4m3_values()[:0x7F]
    x = np.clip(np.asarray(x, dtype=np.float64), -448.0, 448.0)
    a = np.abs(x)
    hi = np.minimum(np.searchsorted(pos, a, side="left"), 0x7E)
    lo = np.maximum(hi - 1, 0)
    dl, dh = a - pos[lo], pos[hi] - a
    pick = np.where(dl < dh, lo, np.where(dh < dl, hi, np.where(lo % 2 == 0, lo, hi)))
    return (pick | np.where(x < 0, 0x80, 0)).astype(np.uint8)


def e4m3_to_f64(c):
    return e4m3_values()[np.asarray(c, dtype=np.int64)]


def subspace_scales_e4m3(X, Ns):
    """One scale per subspace: the largest |x| over the subspace's columns
    divided by 448 (1 where the subspace is all zero).  The scale is an FP32
    number (the quotient rounded to FP32), because the code of every value is
    decided from the FP32 quotient x / scale."""
    X = np.asarray(X, dtype=np.float32)
    d = X.shape[1]
    s = np.empty(Ns, dtype=np.float32)
    for i in range(Ns):
        off, ln = _o.subspace_dims(d, Ns, i)
        m = np.float32(np.abs(X[:, off:off + ln]).max()) if X.shape[0] else np.float32(0.0)
        s[i] = np.float32(m / np.float32(448.0)) if m > 0 else np.float32(1.0)
    return s


def column_scales(scales, d, Ns):
    col = np.empty(d, dtype=np.float64)
    for i in range(Ns):
        off, ln = _o.subspace_dims(d, Ns, i)
        col[off:off + ln] = scales[i]
    return col


def decoded_rows(X, precision, Ns=None, scales=None):
    """Rows as the coarse pass sees them: 1 = BF16, 2 = E4M3 times the
    per-subspace scale."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    if precision == 1:
        return bf16_to_f64(round_bf16(X))
    if precision == 2:
        col32 = column_scales(scales, X.shape[1], Ns).astype(np.float32)
        quot = (X / col32[None, :]).astype(np.float32)  # IEEE FP32 quotient, round to nearest
        return e4m3_to_f64(quantize_e4m3(quot.astype(np.float64))) * col32.astype(np.float64)[None, :]
    raise ValueError(precision)


def coarse_rerank(X, Xhat_rows, q, cands, R, k):
    """Survivors and final top-k of the reduced-precision re-rank.
    Xhat_rows: decoded rows of the candidates (same order as cands)."""
    cands = np.asarray(cands, dtype=np.int64)
    q64 = np.asarray(q, dtype=np.float64)
    coarse = ((np.asarray(Xhat_rows, dtype=np.float64) - q64[None, :]) ** 2).sum(axis=1)
    order = np.lexsort((cands, coarse))
    surv = cands[order[:min(int(R), len(cands))]]
    ids, dist = _o.rerank(X, q, surv, k)
    return dict(survivors=surv, coarse=coarse, coarse_order=order, ids=ids, dist=dist)


def bf16_centroid_tables(index, q):
    """Half-subspace squared distances between the BF16-rounded query and the
    BF16-rounded centroids, in FP64: [Ns][2][sqrtK].  The tensor-core ranking
    computes the same quantity as |q|^2 - 2<q,c> + |c|^2 in FP32."""
    Ns, sk = index["Ns"], index["sqrtK"]
    cent = np.asarray(index["centroids"], dtype=np.float32)
    d = len(q)
    qb = bf16_to_f64(round_bf16(np.asarray(q, dtype=np.float32)))
    out = np.empty((Ns, 2, sk), dtype=np.float64)
    norms = np.empty((Ns, 2, sk), dtype=np.float64)
    for i in range(Ns):
        for h in range(2):
            off, ln = _o.half_dims(d, Ns, i, h)
            cb = bf16_to_f64(round_bf16(cent[i, h, :, :ln]))
            qq = qb[off:off + ln]
            out[i, h] = ((cb - qq[None, :]) ** 2).sum(axis=1)
            norms[i, h] = (qq ** 2).sum() + (cb ** 2).sum(axis=1)
    return out, norms


def fp8_centroid_tables(index, q, data_scales):
    """Half-subspace squared distances between the E4M3-coded query and the
    E4M3-coded centroids, in FP64: [Ns][2][sqrtK], and the norms
    |q_h|^2 + |c|^2 of the coded vectors (the scale of the FP32 error of the
    tensor-core form |q|^2 - 2<q,c> + |c|^2).  Centroids of subspace i are
    coded with the dataset's scale data_scales[i]; the query with its own
    scale t_i = (largest |q| over subspace i) / 448 in FP32 (1 for an all-zero
    subspace); every code is e4m3 of the FP32 quotient, its value code * scale."""
    Ns, sk = index["Ns"], index["sqrtK"]
    cent = np.asarray(index["centroids"], dtype=np.float32)
    q = np.asarray(q, dtype=np.float32)
    d = len(q)
    out = np.empty((Ns, 2, sk), dtype=np.float64)
    norms = np.empty((Ns, 2, sk), dtype=np.float64)
    for i in range(Ns):
        so, sl = _o.subspace_dims(d, Ns, i)
        m = np.float32(np.abs(q[so:so + sl]).max())
        t = np.float32(m / np.float32(448.0)) if m > 0 else np.float32(1.0)
        s = np.float32(data_scales[i])
        for h in range(2):
            off, ln = _o.half_dims(d, Ns, i, h)
            qc = e4m3_to_f64(quantize_e4m3((q[off:off + ln] / t).astype(np.float32).astype(np.float64))) * float(t)
            cc = e4m3_to_f64(quantize_e4m3((cent[i, h, :, :ln] / s).astype(np.float32).astype(np.float64))) * float(s)
            out[i, h] = ((cc - qc[None, :]) ** 2).sum(axis=1)
            norms[i, h] = (qc ** 2).sum() + (cc ** 2).sum(axis=1)
    return out, norms
