"""Seeded synthetic workloads shaped like the paper's datasets.

This module holds only random-number generation and the workload table; it
contains none of the method's arithmetic.  Both the CUDA path's tests and the
CPU oracle draw their inputs from here, and nothing else is shared between them.

The paper's datasets (Table 3: SIFT, GIST, Deep, SPACEV, Turing, TinyImages)
are not available; each generator below stands in for one of them with the
same shape and value type.  Seeds: data 1000+c, queries 2000+c, training
queries 3000+c, K-means initial ids 4000+c (c = workload number).
"""
from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np


@dataclass(frozen=True)
class Workload:
    number: int
    name: str
    n: int
    d: int
    Ns: int
    sqrtK: int
    alpha: float
    beta: float
    k: int
    nq: int
    batch: int
    kmeans_iters: int = 20
    alpha_mix: Tuple[float, ...] = field(default_factory=tuple)
    k_mix: Tuple[int, ...] = field(default_factory=tuple)
    n_train: int = 0
    stands_in_for: str = ""


WORKLOADS = {
    1: Workload(1, "tiny-gaussian-mixture", n=10_000, d=128, Ns=8, sqrtK=10, alpha=0.05, beta=0.005, k=10,
                nq=100, batch=100, stands_in_for="none (small oracle-checkable case)"),
    2: Workload(2, "sift-like-1M", n=1_000_000, d=128, Ns=8, sqrtK=50, alpha=0.05, beta=0.005, k=50,
                nq=10_000, batch=1024, stands_in_for="SIFT (d=128, integer features 0..255)"),
    3: Workload(3, "gist-like-1M", n=1_000_000, d=960, Ns=16, sqrtK=64, alpha=0.03, beta=0.005, k=10,
                nq=10_000, batch=1024, stands_in_for="GIST1M (d=960, non-negative dense)"),
    4: Workload(4, "deep-like-10M", n=10_000_000, d=96, Ns=8, sqrtK=100, alpha=0.05, beta=0.005, k=10,
                nq=100_000, batch=4096, alpha_mix=(0.01, 0.03, 0.05), k_mix=(1, 10, 100),
                stands_in_for="Yandex Deep10M (d=96, unit norm)"),
    5: Workload(5, "hard-mixture-1M", n=1_000_000, d=256, Ns=16, sqrtK=50, alpha=0.05, beta=0.005, k=10,
                nq=10_000, batch=1024, n_train=200_000, stands_in_for="Deep1M shape (d=256), harder mixture"),
}


def _mixture_params(number: int):
    """Per-workload distribution parameters, drawn from the data seed."""
    rng = np.random.default_rng(1000 + number)
    w = WORKLOADS[number]
    if number == 1:
        return dict(centres=rng.uniform(0.0, 100.0, size=(100, w.d)))
    if number == 2:
        return dict(lam=rng.gamma(2.0, 10.0, size=w.d))
    if number == 3:
        return dict()
    if number == 4:
        centres = rng.standard_normal(size=(1000, w.d))
        scales = np.exp(rng.uniform(np.log(0.1), np.log(1.0), size=(1000, w.d)))
        return dict(centres=centres, scales=scales)
    if number == 5:
        centres = rng.uniform(0.0, 100.0, size=(2000, w.d))
        sigma = np.exp(rng.uniform(np.log(0.5), np.log(8.0), size=2000))
        return dict(centres=centres, sigma=sigma, lo=centres.min(axis=0), hi=centres.max(axis=0))
    raise ValueError(number)


def _draw(number: int, rng: np.random.Generator, m: int, params) -> np.ndarray:
    w = WORKLOADS[number]
    d = w.d
    if number == 1:
        lab = rng.integers(0, params["centres"].shape[0], size=m)
        x = params["centres"][lab] + rng.normal(0.0, 5.0, size=(m, d))
    elif number == 2:
        x = np.minimum(rng.poisson(params["lam"][None, :], size=(m, d)), 255)
    elif number == 3:
        x = rng.gamma(1.5, 0.05, size=(m, d))
        x[rng.random(size=(m, d)) < 0.3] = 0.0
    elif number == 4:
        lab = rng.integers(0, params["centres"].shape[0], size=m)
        x = params["centres"][lab] + params["scales"][lab] * rng.standard_normal(size=(m, d))
        x /= np.linalg.norm(x, axis=1, keepdims=True)
    elif number == 5:
        lab = rng.integers(0, params["centres"].shape[0], size=m)
        x = params["centres"][lab] + params["sigma"][lab, None] * rng.standard_normal(size=(m, d))
        noise = rng.random(size=m) < 0.1
        k = int(noise.sum())
        if k:
            x[noise] = params["lo"] + (params["hi"] - params["lo"]) * rng.random(size=(k, d))
    else:
        raise ValueError(number)
    return x.astype(np.float32)


def _generate(number: int, m: int, seed_seq, chunk: int = 1 << 18) -> np.ndarray:
    params = _mixture_params(number)
    out = np.empty((m, WORKLOADS[number].d), dtype=np.float32)
    rng = np.random.default_rng(seed_seq)
    for s in range(0, m, chunk):
        e = min(m, s + chunk)
        out[s:e] = _draw(number, rng, e - s, params)
    return out


def dataset(number: int, n: Optional[int] = None) -> np.ndarray:
    """The n x d float32 dataset of workload `number` (n defaults to the full size)."""
    w = WORKLOADS[number]
    return _generate(number, w.n if n is None else n, [1000 + number, 1])


def queries(number: int, nq: Optional[int] = None, train: bool = False) -> np.ndarray:
    """Fresh draws from the same distribution (never rows of the dataset)."""
    w = WORKLOADS[number]
    m = (w.n_train if train else w.nq) if nq is None else nq
    return _generate(number, m, [(3000 if train else 2000) + number])


def kmeans_init_ids(number: int, n: int, Ns: int, sqrtK: int) -> np.ndarray:
    """[Ns][2][sqrtK] distinct point ids per half-subspace that seed Lloyd's iterations."""
    rng = np.random.default_rng(4000 + number)
    out = np.empty((Ns, 2, sqrtK), dtype=np.int64)
    for i in range(Ns):
        for h in range(2):
            out[i, h] = rng.choice(n, size=sqrtK, replace=False)
    return out


def per_query_mix(number: int, nq: int):
    """Per-query (k, alpha) draws for mixed batches (uniform, independent)."""
    w = WORKLOADS[number]
    rng = np.random.default_rng(5000 + number)
    ks = np.asarray(w.k_mix or (w.k,), dtype=np.int32)
    al = np.asarray(w.alpha_mix or (w.alpha,), dtype=np.float64)
    return ks[rng.integers(0, len(ks), size=nq)], al[rng.integers(0, len(al), size=nq)]


def random_data(seed: int, n: int, d: int, kind: str = "gauss") -> np.ndarray:
    """Small generic inputs for edge-case tests."""
    rng = np.random.default_rng(seed)
    if kind == "gauss":
        return rng.standard_normal(size=(n, d)).astype(np.float32)
    if kind == "int":
        return rng.integers(0, 16, size=(n, d)).astype(np.float32)
    if kind == "uniform":
        return rng.random(size=(n, d)).astype(np.float32)
    raise ValueError(kind)


def random_init_ids(seed: int, n: int, Ns: int, sqrtK: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    out = np.empty((Ns, 2, sqrtK), dtype=np.int64)
    for i in range(Ns):
        for h in range(2):
            out[i, h] = rng.choice(n, size=sqrtK, replace=False)
    return out
