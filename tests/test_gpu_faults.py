"""Failure paths of the C ABI, made on the host (no GPU fault, trap or stall):
an injected allocation failure returns SUCO_ENOMEM and leaks no device memory,
an injected launch failure returns SUCO_ECUDA, and a status word set as if a
bounded device wait had given up is reported by the query entry point as
SUCO_ETIMEOUT until suco_read_status clears it.  After each, the index (or a
new one) answers exactly as before."""
import numpy as np
import pytest
import torch

import paper_2411_14754_gb300 as pkg
from paper_2411_14754_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ENOMEM, ECUDA, ETIMEOUT = -2, -3, -4


@pytest.fixture(scope="module")
def data():
    from paper_2411_14754_gb300 import build
    build.build()
    pkg.load_library()
    X = torch.from_numpy(W.dataset(1, n=4000)).cuda()
    Q = torch.from_numpy(W.queries(1, nq=32)).cuda()
    yield X, Q
    pkg.suco_inject_fault(pkg.FAULT_NONE)


def _free_bytes():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


def _build(X):
    return pkg.suco_build_index(X, 8, 6, 3, seed=11)


def test_every_allocation_of_a_build_fails_cleanly(data):
    X, Q = data
    ref = _build(X)
    want = pkg.suco_query_batch(ref, Q, 10, 0.1, 0.02)
    torch.cuda.synchronize()
    pkg.suco_free(ref)
    base = _free_bytes()
    failures = 0
    for a in range(64):
        pkg.suco_inject_fault(pkg.FAULT_ALLOC, a)
        try:
            ix = _build(X)
        except pkg.SucoError as e:
            assert e.code == ENOMEM, e
            assert _free_bytes() == base, f"allocation {a}: device memory leaked"
            failures += 1
            continue
        pkg.suco_inject_fault(pkg.FAULT_NONE)
        got = pkg.suco_query_batch(ix, Q, 10, 0.1, 0.02)
        torch.cuda.synchronize()
        assert torch.equal(got[0], want[0]) and torch.equal(got[1], want[1])
        pkg.suco_free(ix)
        break
    assert failures >= 10   # index arrays, status word, K-means and IMI scratch
    assert _free_bytes() == base


def test_reduced_copies_allocation_failure_keeps_the_index_usable(data):
    X, Q = data
    ix = _build(X)
    try:
        base = _free_bytes()
        for a in range(3):
            pkg.suco_inject_fault(pkg.FAULT_ALLOC, a)
            with pytest.raises(pkg.SucoError) as e:
                pkg.suco_add_reduced_copies(ix, bf16=False, rank_bf16=False, fp8=True)
            assert e.value.code == ENOMEM
            assert _free_bytes() == base
        pkg.suco_inject_fault(pkg.FAULT_NONE)
        a = pkg.suco_query_batch(ix, Q, 10, 0.1, 0.02)
        pkg.suco_add_reduced_copies(ix)
        b = pkg.suco_query_batch(ix, Q, 10, 0.1, 0.02, precision="fp8", exact_rerank=1000)
        torch.cuda.synchronize()
        assert torch.equal(a[0], b[0])
    finally:
        pkg.suco_inject_fault(pkg.FAULT_NONE)
        pkg.suco_free(ix)


def test_launch_failure_is_reported_and_the_next_call_is_clean(data):
    X, Q = data
    ix = _build(X)
    try:
        want = pkg.suco_query_batch(ix, Q, 10, 0.1, 0.02)
        torch.cuda.synchronize()
        pkg.suco_inject_fault(pkg.FAULT_LAUNCH, 0)
        with pytest.raises(pkg.SucoError) as e:
            pkg.suco_query_batch(ix, Q, 10, 0.1, 0.02)
        assert e.value.code == ECUDA and "injected" in str(e.value)
        got = pkg.suco_query_batch(ix, Q, 10, 0.1, 0.02)
        torch.cuda.synchronize()
        assert torch.equal(got[0], want[0]) and torch.equal(got[1], want[1])
        # a launch failure in the middle of a build: SUCO_ECUDA, nothing leaked
        base = _free_bytes()
        pkg.suco_inject_fault(pkg.FAULT_LAUNCH, 4)
        with pytest.raises(pkg.SucoError) as e:
            _build(X)
        assert e.value.code == ECUDA
        assert _free_bytes() == base
    finally:
        pkg.suco_inject_fault(pkg.FAULT_NONE)
        pkg.suco_free(ix)


def test_a_wait_that_gave_up_is_reported_as_a_timeout(data):
    X, Q = data
    ix = _build(X)
    try:
        pkg.suco_add_reduced_copies(ix)
        want = pkg.suco_query_batch(ix, Q, 10, 0.1, 0.02, rank_precision="bf16")
        torch.cuda.synchronize()
        assert pkg.suco_read_status(ix) == 0
        pkg.suco_inject_fault(pkg.FAULT_WAIT_TIMEOUT, 0)
        with pytest.raises(pkg.SucoError) as e:
            pkg.suco_query_batch(ix, Q, 10, 0.1, 0.02, rank_precision="bf16")
        assert e.value.code == ETIMEOUT
        # the word stays set: every query on the index reports it until it is read
        with pytest.raises(pkg.SucoError) as e:
            pkg.suco_query_batch(ix, Q, 10, 0.1, 0.02)
        assert e.value.code == ETIMEOUT
        assert pkg.suco_read_status(ix) == 1
        assert pkg.suco_read_status(ix) == 0
        got = pkg.suco_query_batch(ix, Q, 10, 0.1, 0.02, rank_precision="bf16")
        torch.cuda.synchronize()
        assert torch.equal(got[0], want[0]) and torch.equal(got[1], want[1])
    finally:
        pkg.suco_inject_fault(pkg.FAULT_NONE)
        pkg.suco_free(ix)
