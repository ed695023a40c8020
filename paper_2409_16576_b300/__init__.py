"""Python binding of libfa, the sm_103a IVF-PQ filtering path of FusionANNS
(arXiv 2409.16576), declared in include/fa.h.

Argument marshalling only: every step of the search runs in the library's
CUDA kernels. The functions carry the C names; numpy arrays are passed as host
buffers and CUDA torch tensors as device buffers (the matching FA_* flags are
set and torch's current stream is used). Importing fails loudly when
``libfa.so`` has not been built (``python paper_2409_16576_b300/_build.py``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfa.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libfa.so is missing: build it with `python paper_2409_16576_b300/_build.py`")

_lib = C.CDLL(LIB_PATH)

# --- enums and flags (include/fa.h) ----------------------------------------
FA_OK, FA_ERR_ARG, FA_ERR_OOM, FA_ERR_CUDA, FA_ERR_TIMEOUT = 0, 1, 2, 3, 4
FA_ERR_OVERFLOW, FA_ERR_STATE, FA_ERR_BUSY, FA_ERR_IO, FA_ERR_NODEV = 5, 6, 7, 8, 9
FA_F32, FA_U8, FA_I8 = 0, 1, 2
FA_RAW_NONE, FA_RAW_HOST_PINNED, FA_RAW_DEVICE, FA_RAW_HOST_PAGED = 0, 1, 2, 3
FA_LUT_F32, FA_LUT_F16, FA_LUT_FP8 = 0, 1, 2
FA_GEMM_SIMT_F32, FA_GEMM_BF16_TC = 0, 1
FA_PROBE_GRAPH = 2  # probe_gemm: the navigation-graph walk
FA_METRIC_L2, FA_METRIC_IP = 0, 1
FA_QUERIES_ON_DEVICE, FA_OUTPUTS_ON_DEVICE, FA_NONBLOCKING = 0x1, 0x2, 0x4
FA_PERSISTENT, FA_NO_SYNC, FA_GRAPH, FA_SERIAL, FA_BATCHED = 0x8, 0x10, 0x20, 0x40, 0x80

P = C.c_void_p
i32, i64, u64, f32 = C.c_int32, C.c_int64, C.c_uint64, C.c_float


class fa_build_params(C.Structure):
    _fields_ = [("nlist", i32), ("M", i32), ("kmeans_iters", i32), ("max_lists_per_vec", i32),
                ("train_sample", i64), ("seed", u64), ("repl_eps", f32), ("raw_location", i32),
                ("use_gpu", i32), ("metric", i32)]


class fa_index_parts(C.Structure):
    _fields_ = [("n", i64), ("d", i32), ("nlist", i32), ("M", i32), ("raw_dtype", i32),
                ("raw_location", i32), ("pad0", i32), ("centroids", P), ("codebooks", P),
                ("codes", P), ("primary", P), ("rep_off", P), ("rep_ids", P), ("raw", P),
                ("metric", i32), ("pad1", i32)]


class fa_index_info(C.Structure):
    _fields_ = [("n", i64), ("n_rep_entries", i64), ("max_list_len", i64), ("max_rep_len", i64),
                ("device_bytes", i64), ("pinned_bytes", i64), ("d", i32), ("nlist", i32),
                ("M", i32), ("device", i32)]


class fa_search_trace(C.Structure):
    _fields_ = [("coarse_ms", f32), ("lut_ms", f32), ("scan_ms", f32), ("post_ms", f32),
                ("total_ms", f32), ("launches", i32), ("handed_back", i32)]


class fa_tune_result(C.Structure):
    _fields_ = [("variants", i32), ("chosen", i32), ("threads", i32 * 8), ("ilp", i32 * 8),
                ("persistent", i32 * 8), ("tile_chunks", i32 * 8), ("ms", f32 * 8)]


class fa_server_params(C.Structure):
    _fields_ = [("max_batch", i32), ("window_us", i32), ("slots", i32), ("kmax", i32),
                ("nprobe_max", i32), ("pad0", i32), ("mem_budget_bytes", i64)]


class fa_server_stats_t(C.Structure):
    _fields_ = [("batches", i64), ("requests", i64), ("pending", i64), ("device_bytes", i64),
                ("inflight_batches", i32), ("slots", i32)]


class fa_search_params(C.Structure):
    _fields_ = [("lut_prec", i32), ("lut_gemm", i32), ("probe_gemm", i32), ("rerank_n", i32),
                ("rerank_batch", i32), ("rerank_beta", i32), ("rerank_eps", f32), ("flags", i32),
                ("k_per_query", P), ("nprobe_per_query", P), ("probes", P), ("stream", P),
                ("stats", P), ("trace", P), ("page_reads", P), ("graph_beam", i32),
                ("graph_max_check", i32), ("graph_entry", i32)]


def _sig(name, res, *args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_sig("fa_build_params_init", None, P)
_sig("fa_search_params_init", None, P)
_sig("fa_build_index", i32, P, i64, i32, i32, P, P)
_sig("fa_index_from_parts", i32, P, P)
_sig("fa_build_index_lists", i32, P, i64, i32, i32, P, i32, P, P, P)
_sig("fa_index_get_parts", i32, P, P)
_sig("fa_index_info_get", i32, P, P)
_sig("fa_save_index", i32, P, C.c_char_p)
_sig("fa_load_index", i32, C.c_char_p, i32, P)
_sig("fa_free_index", None, P)
_sig("fa_search", i32, P, P, i64, i32, i32, i32, P, P)
_sig("fa_search_ex", i32, P, P, i64, i32, i32, i32, P, P, P)
_sig("fa_autotune", i32, P, P, i64, i32, i32, i32, P, P)
_sig("fa_debug_probes", i32, P, P, i64, i32, P, P)
_sig("fa_debug_candidates", i32, P, P, i32, P, P, i64, P)
_sig("fa_debug_lut", i32, P, P, P, P)
_sig("fa_debug_fail_alloc", i32, i32)
_sig("fa_debug_timeout", i32, C.c_uint32)
_sig("fa_debug_tau_sigma", i32, C.c_float)
_sig("fa_debug_page_map", i32, P, P, P, P, P)
_sig("fa_build_probe_graph", i32, P, i32, i32)
_sig("fa_index_get_graph", i32, P, P, P, P, P)
_sig("fa_debug_graph_probe", i32, P, P, i64, i32, i32, i32, i32, P, P, P)
_sig("fa_coarse_probe_noalloc", i32, P, i64, i32, P, i32, i32, P, P)
_sig("fa_server_params_init", None, P)
_sig("fa_server_create", i32, P, P, P, P)
_sig("fa_server_submit", i32, P, P, i64, P, P, P)
_sig("fa_server_poll", i64, P, i64, i32, P, P, P, i32, P, P)
_sig("fa_server_stats", i32, P, P)
_sig("fa_server_destroy", None, P)
_sig("fa_last_error", C.c_char_p)
_sig("fa_status_str", C.c_char_p, i32)
_sig("fa_version", C.c_char_p)

# every symbol include/fa.h declares
EXPORTS = ("fa_build_params_init", "fa_build_index", "fa_build_index_lists", "fa_index_from_parts",
           "fa_index_get_parts",
           "fa_index_info_get", "fa_save_index", "fa_load_index", "fa_free_index",
           "fa_search_params_init", "fa_search", "fa_search_ex", "fa_autotune", "fa_debug_probes",
           "fa_debug_candidates", "fa_debug_lut", "fa_debug_fail_alloc", "fa_debug_timeout",
           "fa_debug_tau_sigma", "fa_debug_page_map", "fa_build_probe_graph", "fa_index_get_graph",
           "fa_debug_graph_probe",
           "fa_coarse_probe_noalloc", "fa_server_params_init",
           "fa_server_create", "fa_server_submit", "fa_server_poll", "fa_server_stats",
           "fa_server_destroy", "fa_last_error",
           "fa_status_str", "fa_version")


class FaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_lib.fa_status_str(status).decode(), msg))
        self.status = status


def _check(st):
    if st != FA_OK:
        raise FaError(st, (_lib.fa_last_error() or b"").decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(P)
    return P(a.data_ptr())  # torch tensor


def _is_cuda(a):
    return a is not None and not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


def fa_version() -> str:
    return _lib.fa_version().decode()


def build_params(**kw) -> fa_build_params:
    p = fa_build_params()
    _lib.fa_build_params_init(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def search_params(**kw) -> fa_search_params:
    p = fa_search_params()
    _lib.fa_search_params_init(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Index:
    """Owns one fa_index handle."""

    def __init__(self, handle):
        self.handle = P(handle)
        self._keep = []

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "handle", None) and self.handle.value:
            _lib.fa_free_index(self.handle)
            self.handle = P(None)

    def info(self) -> fa_index_info:
        out = fa_index_info()
        _check(_lib.fa_index_info_get(self.handle, C.byref(out)))
        return out

    def parts(self, with_raw: bool = True) -> dict:
        """Copies of the logical index (host arrays, caller order); the raw
        vectors only when with_raw."""
        p = fa_index_parts()
        _check(_lib.fa_index_get_parts(self.handle, C.byref(p)))
        n, d, nl, M = p.n, p.d, p.nlist, p.M

        def arr(ptr, dt, shape):
            cnt = int(np.prod(shape))
            if cnt == 0:
                return np.zeros(shape, dtype=dt)
            buf = (C.c_char * (cnt * np.dtype(dt).itemsize)).from_address(ptr)
            return np.frombuffer(buf, dtype=dt).reshape(shape).copy()

        rep_off = arr(p.rep_off, np.int64, (nl + 1,))
        out = dict(n=n, d=d, nlist=nl, M=M, raw_dtype=p.raw_dtype, metric=p.metric,
                   centroids=arr(p.centroids, np.float32, (nl, d)),
                   codebooks=arr(p.codebooks, np.float32, (M, 256, d // M)),
                   codes=arr(p.codes, np.uint8, (n, M)),
                   primary=arr(p.primary, np.int32, (n,)),
                   rep_off=rep_off, rep_ids=arr(p.rep_ids, np.int64, (int(rep_off[-1]),)))
        out["raw"] = arr(p.raw, {FA_U8: np.uint8, FA_I8: np.int8}.get(p.raw_dtype, np.float32), (n, d)) \
            if (p.raw and with_raw) else None
        return out


def _dtype_of(a: np.ndarray) -> int:
    """fa_dtype of a base / raw array: uint8, int8, else float32."""
    if a.dtype == np.uint8:
        return FA_U8
    if a.dtype == np.int8:
        return FA_I8
    return FA_F32


def fa_build_index(base: np.ndarray, params: fa_build_params | None = None) -> Index:
    base = np.ascontiguousarray(base)
    dt = _dtype_of(base)
    if dt == FA_F32:
        base = np.ascontiguousarray(base, dtype=np.float32)
    h = P()
    _check(_lib.fa_build_index(_ptr(base), base.shape[0], base.shape[1], dt,
                               C.byref(params) if params is not None else None, C.byref(h)))
    return Index(h.value)


def fa_build_index_lists(base: np.ndarray, centroids: np.ndarray, primary: np.ndarray,
                         params: fa_build_params | None = None) -> Index:
    """Index over lists the caller already has (PQ trained and encoded here)."""
    base = np.ascontiguousarray(base)
    dt = _dtype_of(base)
    if dt == FA_F32:
        base = np.ascontiguousarray(base, dtype=np.float32)
    cent = np.ascontiguousarray(centroids, dtype=np.float32)
    prim = np.ascontiguousarray(primary, dtype=np.int32)
    h = P()
    _check(_lib.fa_build_index_lists(_ptr(base), base.shape[0], base.shape[1], dt, _ptr(cent),
                                     cent.shape[0], _ptr(prim),
                                     C.byref(params) if params is not None else None, C.byref(h)))
    return Index(h.value)


def fa_index_from_parts(centroids, codebooks, codes, primary, rep_off=None, rep_ids=None,
                        raw=None, raw_location=FA_RAW_HOST_PINNED, metric=FA_METRIC_L2) -> Index:
    cent = np.ascontiguousarray(centroids, dtype=np.float32)
    cb = np.ascontiguousarray(codebooks, dtype=np.float32)
    cd = np.ascontiguousarray(codes, dtype=np.uint8)
    pr = np.ascontiguousarray(primary, dtype=np.int32)
    ro = None if rep_off is None else np.ascontiguousarray(rep_off, dtype=np.int64)
    ri = np.zeros(1, np.int64) if rep_ids is None or len(rep_ids) == 0 else \
        np.ascontiguousarray(rep_ids, dtype=np.int64)
    rw = None if raw is None else np.ascontiguousarray(raw)
    p = fa_index_parts()
    p.n, p.d = cd.shape[0], cent.shape[1]
    p.nlist, p.M = cent.shape[0], cd.shape[1]
    p.raw_dtype = _dtype_of(rw) if rw is not None else FA_F32
    if rw is not None and p.raw_dtype == FA_F32:
        rw = np.ascontiguousarray(rw, dtype=np.float32)
    p.raw_location = raw_location if rw is not None else FA_RAW_NONE
    p.metric = metric
    p.centroids, p.codebooks, p.codes, p.primary = _ptr(cent), _ptr(cb), _ptr(cd), _ptr(pr)
    p.rep_off, p.rep_ids = _ptr(ro), _ptr(ri)
    p.raw = _ptr(rw)
    h = P()
    _check(_lib.fa_index_from_parts(C.byref(p), C.byref(h)))
    return Index(h.value)


def fa_save_index(ix: Index, path: str) -> None:
    _check(_lib.fa_save_index(ix.handle, path.encode()))


def fa_load_index(path: str, raw_location: int = FA_RAW_HOST_PINNED) -> Index:
    h = P()
    _check(_lib.fa_load_index(path.encode(), raw_location, C.byref(h)))
    return Index(h.value)


def fa_search(ix: Index, queries: np.ndarray, k: int, nprobe: int):
    """Plain FP32 form on host buffers: (ids int64 [nq][k], dists float32)."""
    q = np.ascontiguousarray(queries, dtype=np.float32)
    nq, d = q.shape
    ids = np.empty((nq, k), dtype=np.int64)
    dist = np.empty((nq, k), dtype=np.float32)
    _check(_lib.fa_search(ix.handle, _ptr(q), nq, d, k, nprobe, _ptr(ids), _ptr(dist)))
    return ids, dist


def fa_search_ex(ix: Index, queries, k: int, nprobe: int, params: fa_search_params | None = None,
                 out_ids=None, out_dist=None, k_per_query=None, nprobe_per_query=None,
                 probes=None, stats: bool = False, stream=None, trace=None, page_reads=None):
    """Search with explicit parameters. ``queries`` is a float32 numpy array
    (host) or a CUDA torch tensor (device; outputs then default to CUDA
    tensors). Returns (ids, dists) or (ids, dists, stats). ``page_reads``, a
    host int32 array of nq, receives the pages each query's re-rank read
    (raw vectors in FA_RAW_HOST_PAGED)."""
    sp = search_params() if params is None else fa_search_params.from_buffer_copy(params)
    on_dev = _is_cuda(queries)
    keep = []
    if on_dev:
        import torch
        nq, d = queries.shape
        assert queries.dtype == torch.float32 and queries.is_contiguous()
        sp.flags |= FA_QUERIES_ON_DEVICE
        if out_ids is None:
            out_ids = torch.empty((nq, k), dtype=torch.int64, device=queries.device)
            out_dist = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
        if stream is None:
            stream = torch.cuda.current_stream(queries.device).cuda_stream

        def dev_i32(a):
            if a is None:
                return None
            t = a if _is_cuda(a) else torch.as_tensor(np.ascontiguousarray(a, dtype=np.int32),
                                                      device=queries.device)
            keep.append(t)
            return t
        k_per_query, nprobe_per_query, probes = dev_i32(k_per_query), dev_i32(nprobe_per_query), \
            dev_i32(probes)
    else:
        queries = np.ascontiguousarray(queries, dtype=np.float32)
        nq, d = queries.shape
        if out_ids is None:
            out_ids = np.empty((nq, k), dtype=np.int64)
            out_dist = np.empty((nq, k), dtype=np.float32)

        def host_i32(a):
            if a is None:
                return None
            t = np.ascontiguousarray(a, dtype=np.int32)
            keep.append(t)
            return t
        k_per_query, nprobe_per_query, probes = host_i32(k_per_query), host_i32(nprobe_per_query), \
            host_i32(probes)
    if _is_cuda(out_ids):
        sp.flags |= FA_OUTPUTS_ON_DEVICE
    st = np.zeros((nq, 4), dtype=np.int64) if stats else None
    sp.k_per_query, sp.nprobe_per_query, sp.probes = _ptr(k_per_query), _ptr(nprobe_per_query), \
        _ptr(probes)
    sp.stream = stream
    sp.stats = _ptr(st)
    sp.trace = C.cast(C.byref(trace), P) if trace is not None else None
    if page_reads is not None:
        assert page_reads.dtype == np.int32 and page_reads.shape == (nq,) and page_reads.flags.c_contiguous
        sp.page_reads = _ptr(page_reads)
    _check(_lib.fa_search_ex(ix.handle, _ptr(queries), nq, d, k, nprobe, C.byref(sp),
                             _ptr(out_ids), _ptr(out_dist)))
    return (out_ids, out_dist, st) if stats else (out_ids, out_dist)


def fa_autotune(ix: Index, queries: np.ndarray, k: int, nprobe: int, params=None) -> dict:
    """Times the scan's launch shapes on host queries and keeps the fastest in
    the index; returns the timings and the choice."""
    q = np.ascontiguousarray(queries, dtype=np.float32)
    r = fa_tune_result()
    _check(_lib.fa_autotune(ix.handle, _ptr(q), q.shape[0], q.shape[1], k, nprobe,
                            C.byref(params) if params is not None else None, C.byref(r)))
    rows = [dict(threads=r.threads[i], ilp=r.ilp[i], persistent=r.persistent[i],
                 tile_chunks=r.tile_chunks[i], scan_ms=r.ms[i]) for i in range(r.variants)]
    return dict(variants=rows, chosen=rows[r.chosen])


def fa_debug_probes(ix: Index, queries: np.ndarray, nprobe: int, params=None) -> np.ndarray:
    q = np.ascontiguousarray(queries, dtype=np.float32)
    out = np.empty((q.shape[0], nprobe), dtype=np.int32)
    _check(_lib.fa_debug_probes(ix.handle, _ptr(q), q.shape[0], nprobe,
                                C.byref(params) if params is not None else None, _ptr(out)))
    return out


def fa_debug_candidates(ix: Index, query=None, nprobe: int = 1, probes=None, cap=None) -> np.ndarray:
    q = None if query is None else np.ascontiguousarray(query, dtype=np.float32).reshape(-1)
    pr = None if probes is None else np.ascontiguousarray(probes, dtype=np.int32).reshape(-1)
    if pr is not None:
        nprobe = pr.shape[0]
    info = ix.info()
    cap = cap or max(1, (info.max_list_len + info.max_rep_len) * nprobe)
    out = np.empty(cap, dtype=np.int64)
    n = C.c_int64(0)
    _check(_lib.fa_debug_candidates(ix.handle, _ptr(q), nprobe, _ptr(pr), _ptr(out), cap,
                                    C.byref(n)))
    return out[:n.value].copy()


def fa_debug_lut(ix: Index, query, params=None) -> np.ndarray:
    q = np.ascontiguousarray(query, dtype=np.float32).reshape(-1)
    M = ix.info().M
    out = np.empty((M, 256), dtype=np.float32)
    _check(_lib.fa_debug_lut(ix.handle, _ptr(q), C.byref(params) if params is not None else None,
                             _ptr(out)))
    return out


def fa_coarse_probe_noalloc(queries, centroids, nprobe: int, out=None, stream=None, nlist=None):
    """Coarse probe that allocates nothing inside the library, for callers
    that cannot allocate device memory. CUDA torch tensors queries [nq][d] and
    centroids [nlist][d] (float32, contiguous, on one device); output int32
    [nq][nprobe] in ``out`` (a caller that cannot allocate passes its own;
    None lets torch allocate one here). Runs on ``stream`` (default: torch's
    current stream) with the tensors' device current. ``nlist`` overrides the
    row count passed to the C call (used to test its checks; it may only be
    smaller than the centroid rows or rejected by the library before any
    launch). Raises ValueError for tensors the kernels cannot read safely."""
    import torch
    for name, t in (("queries", queries), ("centroids", centroids)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda):
            raise ValueError("%s must be a CUDA tensor" % name)
        if t.dtype != torch.float32 or not t.is_contiguous() or t.dim() != 2:
            raise ValueError("%s must be a contiguous 2-D float32 tensor" % name)
    dev = queries.device
    if centroids.device != dev:
        raise ValueError("queries and centroids must be on the same device")
    nq, d = queries.shape
    if centroids.shape[1] != d:
        raise ValueError("centroids have d=%d, queries d=%d" % (centroids.shape[1], d))
    nl = centroids.shape[0] if nlist is None else int(nlist)
    if nlist is not None and nl > centroids.shape[0] and nl <= (4 << 20):
        # within the library's capacity the kernels would read nl rows
        raise ValueError("nlist above the centroid rows")
    if out is None:
        out = torch.empty((nq, nprobe), dtype=torch.int32, device=dev)
    if not (isinstance(out, torch.Tensor) and out.device == dev and out.dtype == torch.int32
            and out.is_contiguous() and tuple(out.shape) == (nq, nprobe)):
        raise ValueError("out must be a contiguous int32 CUDA tensor of shape (nq, nprobe) "
                         "on the queries' device")
    with torch.cuda.device(dev):
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream
        _check(_lib.fa_coarse_probe_noalloc(_ptr(queries), nq, d, _ptr(centroids), nl, nprobe,
                                            _ptr(out), stream))
    return out


def fa_debug_fail_alloc(n: int) -> None:
    """The n-th next device allocation of the library fails (0 turns it off)."""
    _check(_lib.fa_debug_fail_alloc(n))


def fa_build_probe_graph(ix: Index, R: int = 0, S: int = 0) -> None:
    """Builds the index's navigation graph of lists (§4.1) for FA_PROBE_GRAPH."""
    _check(_lib.fa_build_probe_graph(ix.handle, R, S))


def fa_index_get_graph(ix: Index) -> dict:
    """The navigation graph: adj [nlist][R] (-1 = no edge), seeds [S]."""
    R, S = C.c_int32(0), C.c_int32(0)
    _check(_lib.fa_index_get_graph(ix.handle, None, None, C.byref(R), C.byref(S)))
    adj = np.empty((ix.info().nlist, R.value), dtype=np.int32)
    seeds = np.empty(S.value, dtype=np.int32)
    _check(_lib.fa_index_get_graph(ix.handle, _ptr(adj), _ptr(seeds), None, None))
    return dict(adj=adj, seeds=seeds, R=R.value, S=S.value)


def fa_debug_graph_probe(ix: Index, queries, nprobe: int, beam: int = 0, max_check: int = 0, entry: int = 0):
    """The graph walk alone: (probes [nq][nprobe], -1 past the lists found;
    lists found; vertices checked)."""
    q = np.ascontiguousarray(queries, dtype=np.float32)
    nq = q.shape[0]
    out = np.empty((nq, nprobe), dtype=np.int32)
    found = np.empty(nq, dtype=np.int32)
    checks = np.empty(nq, dtype=np.int32)
    _check(_lib.fa_debug_graph_probe(ix.handle, _ptr(q), nq, nprobe, beam, max_check, entry, _ptr(out),
                                     _ptr(found), _ptr(checks)))
    return out, found, checks


def fa_debug_page_map(ix: Index) -> dict:
    """§4.3's storage layout of paged raw vectors: page and slot of each
    vector (caller ids), rows a page and page count."""
    n = ix.info().n
    page_of = np.empty(n, dtype=np.int64)
    slot_of = np.empty(n, dtype=np.int32)
    rows, pages = C.c_int32(0), C.c_int64(0)
    _check(_lib.fa_debug_page_map(ix.handle, _ptr(page_of), _ptr(slot_of), C.byref(rows), C.byref(pages)))
    return dict(page_of=page_of, slot_of=slot_of, rows_per_page=rows.value, pages=pages.value)


def fa_debug_timeout(polls: int) -> None:
    """Runs a device wait that must run out; raises FaError(FA_ERR_TIMEOUT)."""
    _check(_lib.fa_debug_timeout(polls))


def fa_debug_tau_sigma(sigma: float) -> None:
    """Standard deviations in the scan's sampled threshold estimate (default 4)."""
    _check(_lib.fa_debug_tau_sigma(float(sigma)))


class Server:
    """Request loop with continuous batching (fa_server_*)."""

    def __init__(self, ix: Index, params: fa_search_params | None = None, **kw):
        p = fa_server_params()
        _lib.fa_server_params_init(C.byref(p))
        for key, v in kw.items():
            setattr(p, key, v)
        self.kmax = p.kmax
        self.ix = ix  # keeps the index alive
        h = P()
        _check(_lib.fa_server_create(ix.handle, C.byref(p),
                                     C.byref(params) if params is not None else None, C.byref(h)))
        self.handle = h

    def submit(self, queries, k, nprobe) -> np.ndarray:
        q = np.ascontiguousarray(queries, dtype=np.float32).reshape(-1, queries.shape[-1])
        n = q.shape[0]
        kk = np.ascontiguousarray(np.broadcast_to(k, (n,)), dtype=np.int32)
        nn = np.ascontiguousarray(np.broadcast_to(nprobe, (n,)), dtype=np.int32)
        rid = np.empty(n, dtype=np.int64)
        _check(_lib.fa_server_submit(self.handle, _ptr(q), n, _ptr(kk), _ptr(nn), _ptr(rid)))
        return rid

    def poll(self, max_results=4096, timeout_us=1000):
        rid = np.empty(max_results, dtype=np.int64)
        ids = np.empty((max_results, self.kmax), dtype=np.int64)
        dist = np.empty((max_results, self.kmax), dtype=np.float32)
        lat = np.empty(max_results, dtype=np.float64)
        st = np.empty(max_results, dtype=np.int32)
        n = _lib.fa_server_poll(self.handle, max_results, timeout_us, _ptr(rid), _ptr(ids),
                                _ptr(dist), self.kmax, _ptr(lat), _ptr(st))
        return rid[:n], ids[:n], dist[:n], lat[:n], st[:n]

    def stats(self) -> fa_server_stats_t:
        out = fa_server_stats_t()
        _check(_lib.fa_server_stats(self.handle, C.byref(out)))
        return out

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            _lib.fa_server_destroy(self.handle)
            self.handle = P(None)

    def __del__(self):
        self.close()


def fa_last_error() -> str:
    return (_lib.fa_last_error() or b"").decode()


def fa_status_str(s: int) -> str:
    return _lib.fa_status_str(s).decode()
