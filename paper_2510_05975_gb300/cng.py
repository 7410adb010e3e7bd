"""ctypes binding of libcng.so (include/cng.h): argument marshalling only.

Every function has the C name and forwards to the library; all arithmetic runs in the CUDA
kernels.  PyTorch supplies device memory, streams and views of device arrays.  The library
is loaded on first use; if it has not been built, the call raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcng.so")
_lock = threading.Lock()
_lib = None

CNG_OK, CNG_E_INVAL, CNG_E_NOMEM, CNG_E_CUDA, CNG_E_TIMEOUT, CNG_E_UNSUPPORTED, CNG_E_INTERNAL = (
    0, -1, -2, -3, -4, -5, -6)
CNG_L2, CNG_IP_AS_L2, CNG_IP = 0, 1, 2
CNG_F32, CNG_F16 = 0, 1
CNG_SCREEN_FP32, CNG_SCREEN_TC, CNG_SCREEN_TC_BF16 = 0, 1, 2
CNG_CAND_EXACT, CNG_CAND_BEAM = 0, 1
CNG_SEARCH_FIXED, CNG_SEARCH_LEARNED = 0, 1

EXPORTS = ("cng_build", "cng_free", "cng_last_error", "cng_graph", "cng_lists", "cng_search",
           "cng_knn", "cng_stop_train", "cng_stop_free", "cng_stop_export", "cng_stop_import",
           "cng_trace", "cng_mlp_grad", "cng_mlp_adam", "cng_entry_noalloc", "cng_tune_tau",
           "cngx_wait_probe")
CNG_STOP_NPARAMS = 5313


class CngError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"cng error {code}: {msg}")
        self.code = code


class BuildParams(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("tau", ctypes.c_double), ("R", ctypes.c_int32),
                ("L", ctypes.c_int32), ("metric", ctypes.c_int32), ("screen", ctypes.c_int32),
                ("tie_band", ctypes.c_double), ("margin", ctypes.c_int32),
                ("keep_lists", ctypes.c_int32), ("connect_L", ctypes.c_int32),
                ("input_order", ctypes.c_int32), ("adaptive", ctypes.c_int32),
                ("alpha0", ctypes.c_double), ("alpha_max", ctypes.c_double),
                ("dalpha", ctypes.c_double), ("candidates", ctypes.c_int32),
                ("knn_K", ctypes.c_int32), ("beam_L", ctypes.c_int32),
                ("knn_graph", ctypes.c_void_p), ("repair_slots", ctypes.c_int32),
                ("screen_variant", ctypes.c_int32)]


class BuildStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double) for f in
                ("ms_total", "ms_prep", "ms_entry", "ms_screen", "ms_rerank", "ms_prune", "ms_merge",
                 "ms_connect")] + \
               [(f, ctypes.c_int64) for f in
                ("n_edges", "cert_fail_rows", "order_ties", "rule_ties", "merge_repruned",
                 "merge_max_list", "repair_edges")] + \
               [("repair_rounds", ctypes.c_int32), ("screen_used", ctypes.c_int32),
                ("entry", ctypes.c_int32), ("exact_int", ctypes.c_int32),
                ("screen_err_max", ctypes.c_double), ("ms_order", ctypes.c_double),
                ("alpha_mean", ctypes.c_double), ("ms_cand_search", ctypes.c_double),
                ("screen_variant", ctypes.c_int32), ("screen_stages", ctypes.c_int32),
                ("screen_cap", ctypes.c_int32), ("screen_sync", ctypes.c_int32),
                ("prune_path", ctypes.c_int32)]


class SearchParams(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("model", ctypes.c_void_p), ("threshold", ctypes.c_float),
                ("check_every", ctypes.c_int32), ("max_hops", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("min_stable", ctypes.c_int32)]


class TauTrial(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("L", ctypes.c_int32), ("recall", ctypes.c_double),
                ("hops_mean", ctypes.c_double)]


class SearchStats(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("ndc_total", ctypes.c_int64),
                ("hops_total", ctypes.c_int64), ("fp64_decisions", ctypes.c_int64),
                ("stopped_early", ctypes.c_int64), ("warps_per_block", ctypes.c_int32),
                ("hash_slots", ctypes.c_int32)]


class TrainParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("L", ctypes.c_int32), ("max_trace", ctypes.c_int32),
                ("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("seed", ctypes.c_uint64)]


class TrainStats(ctypes.Structure):
    _fields_ = [("ms_trace", ctypes.c_double), ("ms_train", ctypes.c_double),
                ("samples", ctypes.c_int64), ("positives", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("loss_first", ctypes.c_float), ("loss_last", ctypes.c_float)]


def _as_dict(st) -> dict:
    return {name: getattr(st, name) for name, _ in st._fields_}


def lib():
    """The loaded libcng.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                                   "(there is no fallback implementation)")
            L = ctypes.CDLL(LIB_PATH)
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            L.cng_build.restype = ctypes.c_int
            L.cng_build.argtypes = [vp, i32, i64, i32, ctypes.POINTER(BuildParams), vp,
                                    ctypes.POINTER(vp), ctypes.POINTER(BuildStats)]
            L.cng_free.restype = None
            L.cng_free.argtypes = [vp]
            L.cng_last_error.restype = ctypes.c_char_p
            L.cng_last_error.argtypes = []
            L.cng_graph.restype = ctypes.c_int
            L.cng_graph.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i32),
                                    ctypes.POINTER(i32), ctypes.POINTER(i64)]
            L.cng_lists.restype = ctypes.c_int
            L.cng_lists.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i32),
                                    ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i32)]
            L.cng_search.restype = ctypes.c_int
            L.cng_search.argtypes = [vp, vp, i64, i32, i32, ctypes.POINTER(SearchParams), vp, vp, vp,
                                     vp, vp, vp, ctypes.POINTER(SearchStats)]
            L.cng_knn.restype = ctypes.c_int
            L.cng_knn.argtypes = [vp, i64, vp, i64, i32, i32, i32, ctypes.c_double, vp, vp, vp,
                                  ctypes.POINTER(BuildStats)]
            L.cng_stop_train.restype = ctypes.c_int
            L.cng_stop_train.argtypes = [vp, vp, i64, ctypes.POINTER(TrainParams), vp,
                                         ctypes.POINTER(vp), ctypes.POINTER(TrainStats)]
            L.cng_stop_free.restype = None
            L.cng_stop_free.argtypes = [vp]
            L.cng_stop_export.restype = ctypes.c_int
            L.cng_stop_export.argtypes = [vp, vp, vp, vp, vp]
            L.cng_stop_import.restype = ctypes.c_int
            L.cng_stop_import.argtypes = [vp, vp, vp, ctypes.POINTER(vp)]
            L.cng_trace.restype = ctypes.c_int
            L.cng_trace.argtypes = [vp, vp, i64, i32, i32, i32, vp, vp, vp, vp, vp]
            L.cng_mlp_grad.restype = ctypes.c_int
            L.cng_mlp_grad.argtypes = [vp, vp, vp, i64, vp, vp, vp]
            L.cng_entry_noalloc.restype = ctypes.c_int
            L.cng_entry_noalloc.argtypes = [vp, i32, i64, i32, vp, vp]
            L.cngx_launches.restype = ctypes.c_longlong
            L.cngx_launches.argtypes = []
            L.cng_tune_tau.restype = ctypes.c_int
            L.cng_tune_tau.argtypes = [vp, i32, i64, i32, ctypes.POINTER(BuildParams), vp, i64, i32,
                                       vp, vp, i32, ctypes.c_double, vp,
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(TauTrial),
                                       i32, ctypes.POINTER(ctypes.c_int32)]
            L.cngx_wait_probe.restype = ctypes.c_int
            L.cngx_wait_probe.argtypes = [vp]
            L.cng_mlp_adam.restype = ctypes.c_int
            L.cng_mlp_adam.argtypes = [vp, vp, vp, vp, i64, ctypes.c_float, vp]
            _lib = L
    return _lib


def cngx_wait_probe() -> int:
    """Device status word after the screen's bounded waits were made to run out (include/cng_debug.h)."""
    st = ctypes.c_uint32(0)
    _check(lib().cngx_wait_probe(ctypes.byref(st)))
    return st.value


def cng_last_error() -> str:
    return lib().cng_last_error().decode()


def _check(rc: int):
    if rc != CNG_OK:
        raise CngError(rc, cng_last_error())


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return t.data_ptr()
    return t.ctypes.data  # numpy array (host memory)


class _DevArray:
    """__cuda_array_interface__ view of library-owned device memory."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}


def _view(ptr: int, shape, dtype: torch.dtype) -> torch.Tensor:
    typestr = {torch.int32: "<i4", torch.float32: "<f4"}[dtype]
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device="cuda")


class Index:
    """Owner of a cng_index*; free() releases the device memory."""

    def __init__(self, handle: int, n: int, d: int):
        self.handle, self.n, self.d = handle, n, d

    def free(self):
        if self.handle:
            lib().cng_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def cng_build(points, alpha: float, R: int, L: int, tau: float = 0.0, metric: int = CNG_L2,
              screen: int = CNG_SCREEN_TC, tie_band: float = 1e-5, margin: int = 32,
              keep_lists: bool = False, connect_L: int = 0, input_order: bool = False,
              adaptive=None, candidates: int = 0, knn_K: int = 0, beam_L: int = 0,
              knn_graph: torch.Tensor | None = None, repair_slots: int = 0, screen_variant: int = 0,
              stream=None):
    """cng_build of include/cng.h.  points: CUDA tensor or host (numpy / CPU tensor), float32
    or float16, shape [n, d].  candidates: CNG_CAND_EXACT or CNG_CAND_BEAM (with knn_K,
    beam_L and optionally knn_graph, a CUDA int32 tensor [n, knn_K]).  Returns (Index, stats
    dict)."""
    if isinstance(points, torch.Tensor):
        dt = {torch.float32: CNG_F32, torch.float16: CNG_F16}[points.dtype]
        n, d = points.shape
    else:
        import numpy as np
        dt = {np.dtype("float32"): CNG_F32, np.dtype("float16"): CNG_F16}[points.dtype]
        n, d = points.shape
    a0, am, da = adaptive if adaptive is not None else (0.0, 0.0, 0.0)
    if knn_graph is not None:
        if knn_graph.dtype != torch.int32 or not knn_graph.is_cuda or knn_graph.shape[0] != n:
            raise ValueError("knn_graph must be a CUDA int32 tensor [n, knn_K]")
        knn_K = knn_graph.shape[1]
        knn_graph = knn_graph.contiguous()
    p = BuildParams(alpha, tau, R, L, metric, screen, tie_band, margin, int(keep_lists), connect_L,
                    int(input_order), int(adaptive is not None), a0, am, da, int(candidates),
                    int(knn_K), int(beam_L), None if knn_graph is None else knn_graph.data_ptr(),
                    int(repair_slots), int(screen_variant))
    st = BuildStats()
    h = ctypes.c_void_p()
    _check(lib().cng_build(_ptr(points), dt, n, d, ctypes.byref(p), _stream(stream),
                           ctypes.byref(h), ctypes.byref(st)))
    return Index(h.value, n, d), _as_dict(st)


def cng_tune_tau(points, alpha: float, R: int, L: int, queries, k: int, gt_ids, search_Ls,
                 target: float, metric: int = CNG_L2, screen: int = CNG_SCREEN_TC, stream=None):
    """cng_tune_tau of include/cng.h.  points / queries as cng_build / cng_search; gt_ids: host
    int32 [nq, k].  Returns (best_tau, [dict(tau, L, recall, hops_mean), ...])."""
    import numpy as np
    if isinstance(points, torch.Tensor):
        dt = {torch.float32: CNG_F32, torch.float16: CNG_F16}[points.dtype]
    else:
        dt = {np.dtype("float32"): CNG_F32, np.dtype("float16"): CNG_F16}[points.dtype]
    n, d = points.shape
    p = BuildParams(alpha, 0.0, R, L, metric, screen, 1e-5, 32, 0, 0, 0, 0, 0.0, 0.0, 0.0, 0, 0, 0,
                    None)
    gt = np.ascontiguousarray(gt_ids, dtype=np.int32)
    Ls = np.ascontiguousarray(search_Ls, dtype=np.int32)
    best = ctypes.c_double()
    trials = (TauTrial * 8)()
    nt = ctypes.c_int32()
    _check(lib().cng_tune_tau(_ptr(points), dt, n, d, ctypes.byref(p), _ptr(queries), queries.shape[0],
                              k, gt.ctypes.data, Ls.ctypes.data, len(Ls), float(target), _stream(stream),
                              ctypes.byref(best), trials, 8, ctypes.byref(nt)))
    return best.value, [dict(tau=t.tau, L=t.L, recall=t.recall, hops_mean=t.hops_mean)
                        for t in trials[:nt.value]]


def cng_free(index: Index):
    index.free()


def cng_graph(index: Index):
    """(adj [n, R] int32 view, deg [n] view, R, entry) -- views of library memory."""
    a, dg = ctypes.c_void_p(), ctypes.c_void_p()
    R, e, n = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().cng_graph(index.handle, ctypes.byref(a), ctypes.byref(dg), ctypes.byref(R),
                           ctypes.byref(e), ctypes.byref(n)))
    return (_view(a.value, (n.value, R.value), torch.int32), _view(dg.value, (n.value,), torch.int32),
            R.value, e.value)


def cng_lists(index: Index):
    """(cand [n, L], cdist [n, L], fwd [n, R], fdeg [n]) views; needs keep_lists=True."""
    c, cd, f, fd = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    L, R = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().cng_lists(index.handle, ctypes.byref(c), ctypes.byref(cd), ctypes.byref(L),
                           ctypes.byref(f), ctypes.byref(fd), ctypes.byref(R)))
    n = index.n
    return (_view(c.value, (n, L.value), torch.int32), _view(cd.value, (n, L.value), torch.float32),
            _view(f.value, (n, R.value), torch.int32), _view(fd.value, (n,), torch.int32))


def cng_search(index: Index, queries, k: int, L: int, mode: int = CNG_SEARCH_FIXED, model=None,
               threshold: float = 0.5, check_every: int = 1, max_hops: int = 0,
               use_graph: bool = False, warps_per_block: int = 0, out=None, stream=None,
               with_stats: bool = True, min_stable: int = 0):
    """cng_search of include/cng.h.  queries: CUDA tensor [nq, d] float32 (or host array, then
    outputs are host arrays).  Returns dict(ids, dists, ndc, hops, flags, stats)."""
    nq = queries.shape[0]
    on_dev = isinstance(queries, torch.Tensor) and queries.is_cuda
    if out is None:
        if on_dev:
            dev = queries.device
            out = dict(ids=torch.empty((nq, k), dtype=torch.int32, device=dev),
                       dists=torch.empty((nq, k), dtype=torch.float32, device=dev),
                       ndc=torch.empty(nq, dtype=torch.int32, device=dev),
                       hops=torch.empty(nq, dtype=torch.int32, device=dev),
                       flags=torch.empty(nq, dtype=torch.int32, device=dev))
        else:
            import numpy as np
            out = dict(ids=np.empty((nq, k), np.int32), dists=np.empty((nq, k), np.float32),
                       ndc=np.empty(nq, np.int32), hops=np.empty(nq, np.int32),
                       flags=np.empty(nq, np.int32))
    p = SearchParams(mode, None if model is None else model.handle, threshold, check_every, max_hops,
                     int(use_graph), warps_per_block, int(min_stable))
    st = SearchStats()
    _check(lib().cng_search(index.handle, _ptr(queries), nq, k, L, ctypes.byref(p), _ptr(out["ids"]),
                            _ptr(out["dists"]), _ptr(out.get("ndc")), _ptr(out.get("hops")),
                            _ptr(out.get("flags")), _stream(stream),
                            ctypes.byref(st) if with_stats else None))
    res = dict(out)
    res["stats"] = _as_dict(st) if with_stats else None
    return res


def cng_knn(base: torch.Tensor, k: int, rows: torch.Tensor | None = None,
            screen: int = CNG_SCREEN_TC, tie_band: float = 1e-5, stream=None):
    """cng_knn of include/cng.h: exact (D, id)-ordered k nearest base points per row (CUDA
    float32 tensors).  Returns (ids [m, k] int32, dists [m, k] float32, stats dict)."""
    n, d = base.shape
    m = n if rows is None else rows.shape[0]
    ids = torch.empty((m, k), dtype=torch.int32, device=base.device)
    ds = torch.empty((m, k), dtype=torch.float32, device=base.device)
    st = BuildStats()
    _check(lib().cng_knn(_ptr(base), n, _ptr(rows), m, d, k, screen, tie_band, _ptr(ids), _ptr(ds),
                         _stream(stream), ctypes.byref(st)))
    return ids, ds, _as_dict(st)


class StopModel:
    """Owner of a cng_stop_model*."""

    def __init__(self, handle: int):
        self.handle = handle

    def free(self):
        if self.handle:
            lib().cng_stop_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def cng_stop_train(index: Index, train_queries, k: int, L: int, max_trace: int = 0, epochs: int = 0,
                   batch: int = 0, lr: float = 0.0, seed: int = 1, stream=None):
    """cng_stop_train of include/cng.h; returns (StopModel, stats dict)."""
    p = TrainParams(k, L, max_trace, epochs, batch, lr, seed)
    st = TrainStats()
    h = ctypes.c_void_p()
    _check(lib().cng_stop_train(index.handle, _ptr(train_queries), train_queries.shape[0], ctypes.byref(p),
                                _stream(stream), ctypes.byref(h), ctypes.byref(st)))
    return StopModel(h.value), _as_dict(st)


def cng_stop_free(model: StopModel):
    model.free()


def cng_stop_export(model: StopModel):
    """(params, mu, sigma, bf16-rounded params) as numpy float32 arrays."""
    import numpy as np

    P = np.empty(CNG_STOP_NPARAMS, np.float32)
    mu = np.empty(16, np.float32)
    sg = np.empty(16, np.float32)
    Pb = np.empty(CNG_STOP_NPARAMS, np.float32)
    _check(lib().cng_stop_export(model.handle, _ptr(P), _ptr(mu), _ptr(sg), _ptr(Pb)))
    return P, mu, sg, Pb


def cng_stop_import(params, mu, sigma) -> StopModel:
    import numpy as np

    P = np.ascontiguousarray(params, np.float32)
    m = np.ascontiguousarray(mu, np.float32)
    s_ = np.ascontiguousarray(sigma, np.float32)
    h = ctypes.c_void_p()
    _check(lib().cng_stop_import(_ptr(P), _ptr(m), _ptr(s_), ctypes.byref(h)))
    return StopModel(h.value)


def cng_trace(index: Index, queries: torch.Tensor, k: int, L: int, max_trace: int, stream=None):
    """Per-hop features of the plain search: dict(feats [nq, T, 16], hops, tlc, ids)."""
    nq = queries.shape[0]
    dev = queries.device
    out = dict(feats=torch.full((nq, max_trace, 16), float("nan"), device=dev),
               hops=torch.empty(nq, dtype=torch.int32, device=dev),
               tlc=torch.empty(nq, dtype=torch.int32, device=dev),
               ids=torch.empty((nq, k), dtype=torch.int32, device=dev))
    _check(lib().cng_trace(index.handle, _ptr(queries), nq, k, L, max_trace, _ptr(out["feats"]),
                           _ptr(out["hops"]), _ptr(out["tlc"]), _ptr(out["ids"]), _stream(stream)))
    return out


def cng_mlp_grad(params: torch.Tensor, x: torch.Tensor, y: torch.Tensor, stream=None):
    """(loss, grad) of the stop network's training kernels on one batch (CUDA tensors)."""
    grad = torch.empty(CNG_STOP_NPARAMS, dtype=torch.float32, device=params.device)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    _check(lib().cng_mlp_grad(_ptr(params), _ptr(x), _ptr(y), x.shape[0], _ptr(grad), _ptr(loss),
                              _stream(stream)))
    return loss, grad


def cng_mlp_adam(params: torch.Tensor, m: torch.Tensor, v: torch.Tensor, grad: torch.Tensor, t: int,
                 lr: float, stream=None):
    _check(lib().cng_mlp_adam(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), t, lr, _stream(stream)))


def cng_entry_noalloc(points: torch.Tensor, out: torch.Tensor, stream=None):
    """cng_entry_noalloc of include/cng.h: the navigating node of `points` (CUDA float32 or
    float16 [n, d]) written to `out` (CUDA int32 [1]); allocates nothing."""
    dt = {torch.float32: CNG_F32, torch.float16: CNG_F16}[points.dtype]
    n, d = points.shape
    _check(lib().cng_entry_noalloc(_ptr(points), dt, n, d, _ptr(out), _stream(stream)))
