"""Python binding of ``libsuco`` (the C ABI in ``include/suco.h``).

Argument marshalling only: every step of the query path runs in the CUDA
library.  PyTorch provides device memory and streams.  The functions keep
the C names; see the header for the meaning of each argument.
"""
import ctypes as C
import os
from typing import Optional

import numpy as np
import torch

from . import build as _build

_lib = None


class SucoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libsuco error {code}: {msg}")
        self.code = code


class _BuildParams(C.Structure):
    _fields_ = [("Ns", C.c_int32), ("sqrtK", C.c_int32), ("kmeans_iters", C.c_int32), ("metric", C.c_int32),
                ("seed", C.c_uint64), ("init_ids", C.c_void_p), ("dim_perm", C.c_void_p)]


class _QueryParams(C.Structure):
    _fields_ = [("k", C.c_int32), ("cluster_size", C.c_int32), ("alpha", C.c_double), ("beta", C.c_double),
                ("threads", C.c_int32), ("flags", C.c_int32), ("k_per_query", C.c_void_p),
                ("alpha_per_query", C.c_void_p), ("beta_per_query", C.c_void_p), ("precision", C.c_int32),
                ("exact_rerank", C.c_int32), ("id_passes", C.c_int32), ("rank_precision", C.c_int32)]


class _DebugOut(C.Structure):
    _fields_ = [("t_eff", C.c_void_p), ("activated", C.c_void_p), ("dtab", C.c_void_p), ("scores", C.c_void_p),
                ("cands", C.c_void_p), ("survivors", C.c_void_p), ("stage_clock", C.c_void_p)]


class SucoMlp(C.Structure):
    """ctypes mirror of suco_mlp (device pointers as integers)."""
    _fields_ = [("in_dim", C.c_int32), ("hidden", C.c_int32), ("out_dim", C.c_int32), ("reserved0", C.c_int32),
                ("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p), ("b2", C.c_void_p),
                ("feat_mean", C.c_void_p), ("feat_std", C.c_void_p), ("out_offset", C.c_float * 2),
                ("log_alpha_min", C.c_float), ("log_alpha_max", C.c_float), ("log_beta_min", C.c_float),
                ("log_beta_max", C.c_float), ("fallback_alpha", C.c_float), ("fallback_beta", C.c_float)]


class _IndexInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("Ns", C.c_int32), ("sqrtK", C.c_int32), ("hmax", C.c_int32),
                ("K", C.c_int64), ("ld", C.c_int64), ("device_bytes", C.c_int64), ("metric", C.c_int32),
                ("sampled", C.c_int32)]


def library_path() -> str:
    return _build.LIB


def load_library():
    """Load libsuco.so.  Fails loudly if it has not been built: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2411_14754_gb300.build.build() "
                           "(the SuCo query path has no CPU fallback)")
    L = C.CDLL(path)
    vp, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    L.suco_build_index.argtypes = [vp, i64, i32, C.POINTER(_BuildParams), vp, C.POINTER(vp)]
    L.suco_build_index_from_assignments.argtypes = [vp, i64, i32, i32, i32, vp, vp, vp, C.POINTER(vp)]
    L.suco_build_index_from_parts.argtypes = [vp, i64, i32, C.POINTER(_BuildParams), vp, vp, vp, C.POINTER(vp)]
    L.suco_query_batch.argtypes = [vp, vp, i64, C.POINTER(_QueryParams), vp, vp, vp]
    L.suco_query_debug.argtypes = [vp, vp, i64, C.POINTER(_QueryParams), vp, vp, C.POINTER(_DebugOut), vp]
    L.suco_index_get_info.argtypes = [vp, C.POINTER(_IndexInfo)]
    L.suco_export_index.argtypes = [vp, vp, vp, vp]
    L.suco_thresholds.argtypes = [i64, f64, f64, i32, C.POINTER(i64), C.POINTER(i64)]
    L.suco_kmeans_noalloc.argtypes = [vp, i64, i32, i32, i32, i32, i32, vp, vp, vp]
    L.suco_autotune.argtypes = [vp, vp, i64, C.POINTER(_QueryParams), vp, C.POINTER(i32), C.POINTER(i32)]
    L.suco_query_features.argtypes = [vp, vp, i64, vp, vp]
    L.suco_mlp_predict.argtypes = [vp, C.POINTER(SucoMlp), vp, i64, vp, vp, vp]
    L.suco_mlp_forward.argtypes = [C.POINTER(SucoMlp), vp, i64, vp, vp, vp, vp]
    L.suco_mlp_backward.argtypes = [C.POINTER(SucoMlp), vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.suco_adamw_step.argtypes = [vp, vp, vp, vp, i64, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float,
                                  i32, vp, vp]
    L.suco_add_reduced_copies.argtypes = [vp, i32, vp]
    L.suco_read_status.argtypes = [vp, C.POINTER(C.c_uint32)]
    L.suco_inject_fault.argtypes = [i32, i32]
    L.suco_sc_linear_workspace_size.argtypes = [vp, i64, i32, f64, C.POINTER(C.c_size_t)]
    L.suco_sc_linear.argtypes = [vp, vp, i64, i32, f64, f64, vp, C.c_size_t, vp, vp, vp, vp, vp]
    L.suco_free.argtypes = [vp]
    L.suco_free.restype = None
    L.suco_last_error.restype = C.c_char_p
    for name in ("suco_build_index", "suco_build_index_from_assignments", "suco_build_index_from_parts",
                 "suco_query_batch", "suco_query_debug",
                 "suco_index_get_info", "suco_export_index", "suco_thresholds", "suco_version",
                 "suco_kmeans_noalloc", "suco_autotune", "suco_query_features", "suco_mlp_predict",
                 "suco_mlp_forward", "suco_mlp_backward", "suco_adamw_step", "suco_add_reduced_copies", "suco_read_status",
                 "suco_inject_fault", "suco_sc_linear_workspace_size", "suco_sc_linear"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(rc):
    if rc != 0:
        raise SucoError(rc, load_library().suco_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _same_device(x, ref, name):
    if x.device != ref.device:
        raise ValueError(f"{name} is on {x.device}, the data on {ref.device}")


def _check_assign_out(assign, n, device):
    """An int32 output of n entries that a kernel writes: anything shorter,
    wider, strided or on another device would be written out of bounds."""
    if not isinstance(assign, torch.Tensor) or assign.dtype != torch.int32:
        raise TypeError("assign must be an int32 tensor")
    if not assign.is_contiguous():
        raise ValueError("assign must be contiguous")
    if assign.numel() < n:
        raise ValueError(f"assign holds {assign.numel()} entries, {n} are written")
    if assign.device != device:
        raise ValueError(f"assign is on {assign.device}, the data on {device}")


def _dev_f32(x, name):
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    return x


class SucoIndex:
    """Owns a ``suco_index*``; release it with :func:`suco_free` (or ``with``)."""

    def __init__(self, handle):
        self.handle = handle
        info = _IndexInfo()
        _check(load_library().suco_index_get_info(handle, C.byref(info)))
        self.n, self.d, self.Ns, self.sqrtK = info.n, info.d, info.Ns, info.sqrtK
        self.hmax, self.K, self.ld, self.device_bytes = info.hmax, info.K, info.ld, info.device_bytes
        self.metric, self.sampled = info.metric, info.sampled

    def __enter__(self):
        return self

    def __exit__(self, *a):
        suco_free(self)

    def __del__(self):
        try:
            suco_free(self)
        except Exception:
            pass


METRIC = {"l2": 0, "l1": 1}


def _perm_arg(dim_perm):
    return None if dim_perm is None else np.ascontiguousarray(dim_perm, dtype=np.int32)


def suco_build_index(data: torch.Tensor, Ns: int, sqrtK: int, kmeans_iters: int = 20, seed: int = 0,
                     init_ids: Optional[np.ndarray] = None, stream=None, metric="l2", dim_perm=None) -> SucoIndex:
    """Algorithm 2 on the GPU.  ``data``: n x d float32 CUDA tensor (copied).
    metric "l2" (squared Euclidean) or "l1"; dim_perm: Definition 3's subspace
    sampling as a permutation of the d dims (None: contiguous subspaces)."""
    _dev_f32(data, "data")
    ids = None if init_ids is None else np.ascontiguousarray(init_ids, dtype=np.int64)
    pm = _perm_arg(dim_perm)
    p = _BuildParams(Ns, sqrtK, kmeans_iters, METRIC[metric] if isinstance(metric, str) else int(metric), seed,
                     None if ids is None else ids.ctypes.data, None if pm is None else pm.ctypes.data)
    h = C.c_void_p()
    _check(load_library().suco_build_index(_ptr(data), data.shape[0], data.shape[1], C.byref(p), _stream(stream),
                                           C.byref(h)))
    return SucoIndex(h)


def suco_build_index_from_assignments(data: torch.Tensor, Ns: int, sqrtK: int, centroids, assign,
                                      stream=None) -> SucoIndex:
    """IMI from given centroids [Ns][2][sqrtK][hmax] and assignments [Ns][2][n] (host arrays)."""
    _dev_f32(data, "data")
    cent = np.ascontiguousarray(centroids, dtype=np.float32)
    asg = np.ascontiguousarray(assign, dtype=np.int32)
    h = C.c_void_p()
    _check(load_library().suco_build_index_from_assignments(_ptr(data), data.shape[0], data.shape[1], Ns, sqrtK,
                                                            cent.ctypes.data, asg.ctypes.data, _stream(stream),
                                                            C.byref(h)))
    return SucoIndex(h)


def suco_build_index_from_parts(data: torch.Tensor, Ns: int, sqrtK: int, centroids, assign, metric="l2",
                                dim_perm=None, stream=None) -> SucoIndex:
    """The IMI from given centroids [Ns][2][sqrtK][hmax] (over each half's dims
    in the sampling's order) and assignments [Ns][2][n], for any metric and
    subspace sampling."""
    _dev_f32(data, "data")
    cent = np.ascontiguousarray(centroids, dtype=np.float32)
    asg = np.ascontiguousarray(assign, dtype=np.int32)
    pm = _perm_arg(dim_perm)
    p = _BuildParams(Ns, sqrtK, 0, METRIC[metric] if isinstance(metric, str) else int(metric), 0, None,
                     None if pm is None else pm.ctypes.data)
    h = C.c_void_p()
    _check(load_library().suco_build_index_from_parts(_ptr(data), data.shape[0], data.shape[1], C.byref(p),
                                                      cent.ctypes.data, asg.ctypes.data, _stream(stream), C.byref(h)))
    return SucoIndex(h)


def _per_query(t, dtype, nq, name):
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous() and t.numel() == nq):
        raise TypeError(f"{name} must be a contiguous CUDA tensor of {nq} {dtype}")
    return t.data_ptr()


QUERY_ONE_CLUSTER_PER_QUERY = 1


PRECISION = {"fp32": 0, "bf16": 1, "fp8": 2}  # also the rank_precision codes (SUCO_RANK_*)
COPY_BF16, COPY_RANK_BF16, COPY_FP8 = 1, 2, 4


def _qparams(k, alpha, beta, cluster_size, threads, nq=0, k_per_query=None, alpha_per_query=None,
             beta_per_query=None, flags=0, precision="fp32", exact_rerank=0, id_passes=0, rank_precision="fp32"):
    return _QueryParams(int(k), int(cluster_size), float(alpha), float(beta), int(threads), int(flags),
                        _per_query(k_per_query, torch.int32, nq, "k_per_query"),
                        _per_query(alpha_per_query, torch.float32, nq, "alpha_per_query"),
                        _per_query(beta_per_query, torch.float32, nq, "beta_per_query"),
                        PRECISION[precision] if isinstance(precision, str) else int(precision), int(exact_rerank),
                        int(id_passes), PRECISION[rank_precision] if isinstance(rank_precision, str)
                        else int(rank_precision))


def suco_add_reduced_copies(index: "SucoIndex", bf16: bool = True, rank_bf16: bool = True, fp8: bool = True,
                            stream=None):
    """Add the BF16 and FP8 copies of the index's dataset (precision="bf16" /
    "fp8") and the workspace of the BF16 tensor-core ranking (rank_precision="bf16")."""
    mask = (COPY_BF16 if bf16 else 0) | (COPY_RANK_BF16 if rank_bf16 else 0) | (COPY_FP8 if fp8 else 0)
    _check(load_library().suco_add_reduced_copies(index.handle, mask, _stream(stream)))


def suco_query_batch(index: SucoIndex, queries: torch.Tensor, k: int, alpha: float, beta: float,
                     out_ids: Optional[torch.Tensor] = None, out_dist: Optional[torch.Tensor] = None,
                     cluster_size: int = 0, threads: int = 0, stream=None, k_per_query=None, alpha_per_query=None,
                     beta_per_query=None, flags: int = 0, precision="fp32", exact_rerank: int = 0,
                     id_passes: int = 0, rank_precision="fp32"):
    """Algorithm 4 for every row of ``queries``; returns (ids int32 [nq,k], squared dists float32 [nq,k]).
    Optional per-query CUDA tensors: k_per_query (int32), alpha_per_query, beta_per_query (float32).
    precision "bf16" re-ranks a coarse BF16 pass's exact_rerank survivors (0 = 512) exactly."""
    _dev_f32(queries, "queries")
    nq = queries.shape[0]
    if out_ids is None:
        out_ids = torch.empty((nq, k), dtype=torch.int32, device=queries.device)
    if out_dist is None:
        out_dist = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
    p = _qparams(k, alpha, beta, cluster_size, threads, nq, k_per_query, alpha_per_query, beta_per_query, flags,
                 precision, exact_rerank, id_passes, rank_precision)
    _check(load_library().suco_query_batch(index.handle, _ptr(queries), nq, C.byref(p), _ptr(out_ids),
                                           _ptr(out_dist), _stream(stream)))
    return out_ids, out_dist


def suco_query_debug(index: SucoIndex, queries: torch.Tensor, k: int, alpha: float, beta: float,
                     cluster_size: int = 0, threads: int = 0, want=("t_eff", "activated", "dtab", "scores", "cands"),
                     stream=None, k_per_query=None, alpha_per_query=None, beta_per_query=None, flags: int = 0,
                     precision="fp32", exact_rerank: int = 0, id_passes: int = 0, rank_precision="fp32"):
    """suco_query_batch plus per-stage outputs; returns a dict of CUDA tensors."""
    _dev_f32(queries, "queries")
    nq = queries.shape[0]
    dev = queries.device
    T, Cc = suco_thresholds(index.n, alpha, beta, k)
    out = dict(ids=torch.empty((nq, k), dtype=torch.int32, device=dev),
               dist=torch.empty((nq, k), dtype=torch.float32, device=dev))
    shapes = dict(t_eff=((nq, index.Ns), torch.int64), activated=((nq, index.Ns, index.K), torch.uint8),
                  dtab=((nq, index.Ns, 2, index.sqrtK), torch.float32), scores=((nq, index.n), torch.uint8),
                  cands=((nq, Cc), torch.int32), survivors=((nq, index.n), torch.uint8),
                  stage_clock=((nq, 16, 20), torch.int64))
    for name in want:
        shp, dt = shapes[name]
        fill = 0 if name == "survivors" else (-1 if dt != torch.uint8 else 255)
        out[name] = torch.full(shp, fill, dtype=dt, device=dev)
    dbg = _DebugOut(*[(out[n].data_ptr() if n in out else None) for n in ("t_eff", "activated", "dtab", "scores",
                                                                        "cands", "survivors", "stage_clock")])
    p = _qparams(k, alpha, beta, cluster_size, threads, nq, k_per_query, alpha_per_query, beta_per_query, flags,
                 precision, exact_rerank, id_passes, rank_precision)
    _check(load_library().suco_query_debug(index.handle, _ptr(queries), nq, C.byref(p), _ptr(out["ids"]),
                                           _ptr(out["dist"]), C.byref(dbg), _stream(stream)))
    out["T"], out["C"] = T, Cc
    return out


def suco_autotune(index: SucoIndex, queries: torch.Tensor, k: int, alpha: float, beta: float, stream=None,
                  k_per_query=None, alpha_per_query=None, beta_per_query=None, flags: int = 0):
    """Time every launch shape on these queries; the index remembers the fastest.
    Returns (cluster_size, threads)."""
    _dev_f32(queries, "queries")
    nq = queries.shape[0]
    p = _qparams(k, alpha, beta, 0, 0, nq, k_per_query, alpha_per_query, beta_per_query, flags)
    cl, nt = C.c_int32(), C.c_int32()
    _check(load_library().suco_autotune(index.handle, _ptr(queries), nq, C.byref(p), _stream(stream), C.byref(cl),
                                        C.byref(nt)))
    return cl.value, nt.value


def suco_query_features(index: SucoIndex, queries: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None):
    """Per-query features [nq][3*Ns] (see include/suco.h)."""
    _dev_f32(queries, "queries")
    nq = queries.shape[0]
    if out is None:
        out = torch.empty((nq, 3 * index.Ns), dtype=torch.float32, device=queries.device)
    _check(load_library().suco_query_features(index.handle, _ptr(queries), nq, _ptr(out), _stream(stream)))
    return out


def suco_mlp_predict(index: SucoIndex, model: SucoMlp, queries: torch.Tensor, alpha: Optional[torch.Tensor] = None,
                     beta: Optional[torch.Tensor] = None, stream=None):
    """Per-query (alpha, beta) float32 CUDA tensors from the network."""
    _dev_f32(queries, "queries")
    nq = queries.shape[0]
    if alpha is None:
        alpha = torch.empty(nq, dtype=torch.float32, device=queries.device)
    if beta is None:
        beta = torch.empty(nq, dtype=torch.float32, device=queries.device)
    _check(load_library().suco_mlp_predict(index.handle, C.byref(model), _ptr(queries), nq, _ptr(alpha), _ptr(beta),
                                           _stream(stream)))
    return alpha, beta


def suco_mlp_forward(model: SucoMlp, x: torch.Tensor, z1=None, h=None, y=None, stream=None):
    _dev_f32(x, "x")
    B = x.shape[0]
    if y is None:
        y = torch.empty((B, 2), dtype=torch.float32, device=x.device)
    _check(load_library().suco_mlp_forward(C.byref(model), _ptr(x), B, _ptr(z1), _ptr(h), _ptr(y), _stream(stream)))
    return y


def suco_mlp_backward(model: SucoMlp, x, z1, h, y, target, dz1, dy, dw1, db1, dw2, db2, loss, stream=None):
    _check(load_library().suco_mlp_backward(C.byref(model), _ptr(x), x.shape[0], _ptr(z1), _ptr(h), _ptr(y),
                                            _ptr(target), _ptr(dz1), _ptr(dy), _ptr(dw1), _ptr(db1), _ptr(dw2),
                                            _ptr(db2), _ptr(loss), _stream(stream)))


def suco_adamw_step(param, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0,
                    bf16_copy=None, stream=None):
    _check(load_library().suco_adamw_step(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), lr, beta1, beta2,
                                          eps, weight_decay, int(step), _ptr(bf16_copy), _stream(stream)))


def suco_index_get_info(index: SucoIndex) -> dict:
    return dict(n=index.n, d=index.d, Ns=index.Ns, sqrtK=index.sqrtK, hmax=index.hmax, K=index.K, ld=index.ld,
                device_bytes=index.device_bytes)


def suco_export_index(index: SucoIndex) -> dict:
    cent = np.empty((index.Ns, 2, index.sqrtK, index.hmax), dtype=np.float32)
    off = np.empty((index.Ns, index.K + 1), dtype=np.uint32)
    perm = np.empty((index.Ns, index.n), dtype=np.int32)
    _check(load_library().suco_export_index(index.handle, cent.ctypes.data, off.ctypes.data, perm.ctypes.data))
    return dict(centroids=cent, cell_off=off, perm=perm)


def suco_thresholds(n: int, alpha: float, beta: float, k: int):
    T, Cc = C.c_int64(), C.c_int64()
    _check(load_library().suco_thresholds(int(n), float(alpha), float(beta), int(k), C.byref(T), C.byref(Cc)))
    return T.value, Cc.value


def suco_kmeans_noalloc(data: torch.Tensor, dim_off: int, dim_len: int, centroids: torch.Tensor, iters: int,
                        assign: torch.Tensor = None, stream=None):
    """Lloyd K-means on columns [dim_off, dim_off+dim_len) of ``data`` without any
    device allocation inside the library.  ``centroids`` (k x dim_len float32
    CUDA tensor) holds the initial centroids and receives the final ones;
    returns the int32 assignment (written into ``assign`` if given)."""
    _dev_f32(data, "data")
    _dev_f32(centroids, "centroids")
    n, d = data.shape
    k = centroids.shape[0]
    if centroids.dim() != 2 or centroids.shape[1] != dim_len:
        raise ValueError("centroids must be k x dim_len")
    _same_device(centroids, data, "centroids")
    if assign is None:
        assign = torch.empty(n, dtype=torch.int32, device=data.device)
    else:
        _check_assign_out(assign, n, data.device)
    _check(load_library().suco_kmeans_noalloc(_ptr(data), n, d, dim_off, dim_len, k, iters, _ptr(centroids),
                                              _ptr(assign), _stream(stream)))
    return assign


def suco_sc_linear_workspace_size(index: SucoIndex, batch: int, k: int, beta: float) -> int:
    nb = C.c_size_t()
    _check(load_library().suco_sc_linear_workspace_size(index.handle, int(batch), int(k), float(beta), C.byref(nb)))
    return nb.value


def suco_sc_linear(index: SucoIndex, queries: torch.Tensor, k: int, alpha: float, beta: float,
                   workspace: Optional[torch.Tensor] = None, batch: int = 32, out_ids=None, out_dist=None,
                   debug: bool = False, stream=None):
    """SC-Linear (Algorithm 1) for every row of ``queries``.  ``workspace``: a
    uint8 CUDA tensor (allocated for ``batch`` queries when not given).
    Returns (ids, dists) or, with debug, (ids, dists, scores [nq][n] uint8,
    cands [nq][C] int32)."""
    _dev_f32(queries, "queries")
    nq = queries.shape[0]
    dev = queries.device
    if workspace is None:
        nb = suco_sc_linear_workspace_size(index, max(1, min(batch, nq)), k, beta)
        workspace = torch.empty(nb, dtype=torch.uint8, device=dev)
    if out_ids is None:
        out_ids = torch.empty((nq, k), dtype=torch.int32, device=dev)
    if out_dist is None:
        out_dist = torch.empty((nq, k), dtype=torch.float32, device=dev)
    sc = cd = None
    if debug:
        _, Cc = suco_thresholds(index.n, alpha, beta, k)
        sc = torch.full((nq, index.n), 255, dtype=torch.uint8, device=dev)
        cd = torch.full((nq, Cc), -1, dtype=torch.int32, device=dev)
    _check(load_library().suco_sc_linear(index.handle, _ptr(queries), nq, int(k), float(alpha), float(beta),
                                         _ptr(workspace), workspace.numel(), _ptr(out_ids), _ptr(out_dist), _ptr(sc),
                                         _ptr(cd), _stream(stream)))
    return (out_ids, out_dist, sc, cd) if debug else (out_ids, out_dist)


def suco_free(index: SucoIndex):
    if index is not None and index.handle:
        load_library().suco_free(index.handle)
        index.handle = None


def suco_read_status(index: SucoIndex) -> int:
    """Read and clear the index's device status word (0: every launch completed normally)."""
    st = C.c_uint32(0)
    _check(load_library().suco_read_status(index.handle, C.byref(st)))
    return int(st.value)


FAULT_NONE, FAULT_ALLOC, FAULT_LAUNCH, FAULT_WAIT_TIMEOUT = 0, 1, 2, 3


def suco_inject_fault(kind: int, after: int = 0):
    """Arm one host-side fault (test hook): the after-th allocation, kernel
    launch or tensor-core ranking wait from now fails (see include/suco.h)."""
    _check(load_library().suco_inject_fault(int(kind), int(after)))


def suco_last_error() -> str:
    return load_library().suco_last_error().decode()


def suco_version() -> int:
    return load_library().suco_version()
