"""The C-ABI library loads without a GPU and exports every declared entry point;
host-only logic (thresholds, argument checks that need no device) is checked here."""
import ctypes
import os
import re

import pytest

import oracle
from paper_2411_14754_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "suco.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(suco_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("suco_build_index", "suco_query_batch", "suco_free"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_exports_nothing_else():
    out = os.popen(f"nm -D --defined-only {B.LIB}").read()
    exported = sorted(set(re.findall(r" T (suco_\w+)", out)))
    assert exported == declared_functions()


def test_library_is_built_for_sm_103a_only():
    out = os.popen(f"cuobjdump --list-elf {B.LIB} 2>/dev/null").read()
    archs = set(re.findall(r"sm_\w+", out))
    assert archs == {"sm_103a"}, archs


@pytest.mark.parametrize("n,alpha,beta,k", [(10_000, 0.05, 0.005, 10), (1_000_000, 0.05, 0.005, 50),
                                            (100, 0.07, 0.001, 10), (5, 0.5, 0.5, 10), (123, 1.0, 1.0, 1),
                                            (10_000_000, 0.03, 0.003, 100), (7, 1e-9, 1e-9, 3)])
def test_thresholds_agree_with_the_oracle_reading(lib, n, alpha, beta, k):
    T, C = ctypes.c_int64(), ctypes.c_int64()
    lib.suco_thresholds.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    assert lib.suco_thresholds(n, alpha, beta, k, ctypes.byref(T), ctypes.byref(C)) == 0
    assert T.value == oracle.collision_threshold(alpha, n)
    assert C.value == oracle.candidate_count(beta, n, k)


def test_host_side_argument_errors(lib):
    lib.suco_last_error.restype = ctypes.c_char_p
    lib.suco_thresholds.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                    ctypes.c_void_p, ctypes.c_void_p]
    assert lib.suco_thresholds(10, 0.1, 0.1, 1, None, None) == -1
    assert b"NULL" in lib.suco_last_error()
    T, C = ctypes.c_int64(), ctypes.c_int64()
    assert lib.suco_thresholds(10, 0.0, 0.1, 1, ctypes.byref(T), ctypes.byref(C)) == -1
    assert lib.suco_thresholds(10, 0.1, 1.5, 1, ctypes.byref(T), ctypes.byref(C)) == -1
    lib.suco_build_index.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]
    assert lib.suco_build_index(None, 10, 16, None, None, None) == -1
    lib.suco_query_batch.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int64] + [ctypes.c_void_p] * 4
    assert lib.suco_query_batch(None, None, 1, None, None, None, None) == -1
    lib.suco_free.argtypes = [ctypes.c_void_p]
    lib.suco_free(None)  # NULL-safe
    assert lib.suco_version() == 100


def test_noalloc_assign_output_is_checked_before_any_launch():
    # the K-means kernel writes n int32 values into assign: a tensor that is
    # short, of another type, strided or on another device is refused on the host
    torch = pytest.importorskip("torch")
    from paper_2411_14754_gb300 import suco as S
    cpu = torch.device("cpu")
    S._check_assign_out(torch.empty(10, dtype=torch.int32), 10, cpu)
    S._check_assign_out(torch.empty(12, dtype=torch.int32), 10, cpu)
    with pytest.raises(TypeError):
        S._check_assign_out(torch.empty(10, dtype=torch.int16), 10, cpu)
    with pytest.raises(TypeError):
        S._check_assign_out(torch.empty(10, dtype=torch.int64), 10, cpu)
    with pytest.raises(TypeError):
        S._check_assign_out(None, 10, cpu)
    with pytest.raises(ValueError):
        S._check_assign_out(torch.empty(9, dtype=torch.int32), 10, cpu)
    with pytest.raises(ValueError):
        S._check_assign_out(torch.empty(20, dtype=torch.int32)[::2], 10, cpu)
    with pytest.raises(ValueError):
        S._check_assign_out(torch.empty(10, dtype=torch.int32, device="meta"), 10, cpu)
    with pytest.raises(ValueError):
        S._same_device(torch.empty(3, device="meta"), torch.empty(3), "centroids")
    S._same_device(torch.empty(3), torch.empty(3), "centroids")


def test_fault_injection_on_the_host_without_a_gpu(lib):
    # an injected failure of the host index allocation is reported before the
    # library touches the device: suco_build_index returns SUCO_ENOMEM
    lib.suco_last_error.restype = ctypes.c_char_p
    lib.suco_inject_fault.argtypes = [ctypes.c_int32, ctypes.c_int32]
    assert lib.suco_inject_fault(9, 0) == -1
    assert lib.suco_inject_fault(1, -1) == -1

    class Params(ctypes.Structure):
        _fields_ = [("Ns", ctypes.c_int32), ("sqrtK", ctypes.c_int32), ("kmeans_iters", ctypes.c_int32),
                    ("metric", ctypes.c_int32), ("seed", ctypes.c_uint64), ("init_ids", ctypes.c_void_p),
                    ("dim_perm", ctypes.c_void_p)]

    lib.suco_build_index.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Params),
                                     ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    out = ctypes.c_void_p()
    p = Params(2, 4, 1, 0, 7, None, None)
    assert lib.suco_inject_fault(1, 0) == 0                       # SUCO_FAULT_ALLOC, the next allocation
    rc = lib.suco_build_index(ctypes.c_void_p(16), 100, 8, ctypes.byref(p), None, ctypes.byref(out))
    assert rc == -2 and out.value is None
    assert b"injected" in lib.suco_last_error() or b"host allocation" in lib.suco_last_error()
    assert lib.suco_inject_fault(0, 0) == 0                       # disarm
