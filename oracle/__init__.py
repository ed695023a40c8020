"""FP64 CPU oracle for the IVF-PQ filtering path (FusionANNS, arXiv 2409.16576).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package. It shares no code with
the CUDA path (``paper_2409_16576_b300``) and neither imports the other.

The arithmetic lives in ``oracle.c`` (plain C, double precision, OpenMP over
queries); this module compiles it with gcc and marshals numpy arrays. Each C
function cites the step of the paper it follows:

  ``coarse``      step 2 of §3, exact top-nprobe lists (pinned: brute force
                  against scipy's cdist, self-probe invariant)
  ``lut``         step 1 / the dist() terms of Eq. 1 (pinned: scipy cdist per
                  subspace, hand-worked golden table)
  ``candidates``  steps 3-5, gather + sort-unique (pinned: unique count = N
                  and gathered = sum of list sizes at nprobe = nlist)
  ``adc``         step 6, Eq. 1 (pinned: identity codebook gives exact L2)
  ``topn``        step 7 (pinned: numpy lexsort)
  ``rerank``      step 8, Algorithm 1 + Eq. 3 (pinned: eps<0 gives the exact
                  top-k of the n candidates; beta=1, eps>=1 stops after the
                  first mini-batch; a hand-worked Delta sequence)
  ``search``      the pipeline (pinned: identity codebook + nprobe = nlist
                  equals brute-force k-NN)
  ``knn``         brute-force ground truth (pinned: numpy on tiny inputs)

Every step also takes ``metric=IP`` (the negated inner product -<q, x>, the
second metric of the SPACEV-like workload) and int8 raw rows; those forms are
pinned against numpy inner products, an identity codebook and brute force.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

RAW_F32 = 0
RAW_U8 = 1
RAW_I8 = 2

L2 = 0   # squared L2 distance
IP = 1   # negated inner product: -<q, x> (smallest first)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        i32, i64, f32 = C.c_int32, C.c_int64, C.c_float
        _lib.or_coarse.argtypes = [P, i64, i32, P, i32, i32, P, P]
        _lib.or_lut.argtypes = [P, i32, i32, P, P]
        _lib.or_candidates.argtypes = [P, i32, P, P, P, i64, P]
        _lib.or_candidates.restype = i64
        _lib.or_adc.argtypes = [P, i32, P, P, i64, P]
        _lib.or_topn.argtypes = [P, P, i64, i32, P, P]
        _lib.or_exact_l2.argtypes = [P, i32, P, i32, P, i64, P]
        _lib.or_rerank.argtypes = [P, i32, P, i32, P, i32, i32, i32, f32, i32, P, P]
        _lib.or_rerank.restype = i32
        _lib.or_search.argtypes = [P, i64, i32, P, i32, i32, P, P, P, P, P, i32, i32, i32, P,
                                   i32, i32, f32, i32, P, P, P]
        _lib.or_search.restype = i32
        _lib.or_knn.argtypes = [P, i64, P, i32, i64, i32, i32, P, P]
        _lib.or_num_threads.restype = i32
        _lib.or_set_threads.argtypes = [i32]
        _lib.or_coarse_m.argtypes = [P, i64, i32, P, i32, i32, P, P, i32]
        _lib.or_lut_m.argtypes = [P, i32, i32, P, P, i32]
        _lib.or_exact_m.argtypes = [P, i32, P, i32, P, i64, P, i32]
        _lib.or_rerank_m.argtypes = [P, i32, P, i32, P, i32, i32, i32, f32, i32, P, P, i32]
        _lib.or_rerank_m.restype = i32
        _lib.or_search_m.argtypes = [P, i64, i32, P, i32, i32, P, P, P, P, P, i32, i32, i32, P,
                                     i32, i32, f32, i32, P, P, P, i32]
        _lib.or_search_m.restype = i32
        _lib.or_knn_m.argtypes = [P, i64, P, i32, i64, i32, i32, P, P, i32]
        _lib.or_page_layout.argtypes = [P, i64, i32, i32, P, P]
        _lib.or_page_layout.restype = i64
        _lib.or_rerank_pages.argtypes = [P, i32, P, i32, P, i32, i32, i32, f32, i32, P, P, P, i32, P]
        _lib.or_rerank_pages.restype = i32
        _lib.or_graph_probe.argtypes = [P, i64, i32, P, i32, P, i32, P, i32, i32, i32, i32, i32, i32, P, P, P]
        _lib.or_graph_heads.argtypes = [P, i32, i32, i32, P]
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def num_threads() -> int:
    return lib().or_num_threads()


def set_threads(t: int) -> None:
    lib().or_set_threads(int(t))


def raw_kind(raw: np.ndarray) -> int:
    if raw.dtype == np.uint8:
        return RAW_U8
    if raw.dtype == np.int8:
        return RAW_I8
    return RAW_F32


# ---------------------------------------------------------------------------
# logical index helpers
# ---------------------------------------------------------------------------

def lists_from_parts(primary, rep_off, rep_ids, nlist):
    """Plain posting lists (CSR of vector ids) from the primary list of each
    vector plus per-list replica ids: list l = {v : primary[v] = l} followed
    by rep_ids[rep_off[l]:rep_off[l+1]]."""
    primary = np.asarray(primary, dtype=np.int64)
    order = np.argsort(primary, kind="stable")
    counts = np.bincount(primary, minlength=nlist)
    rep_off = np.asarray(rep_off, dtype=np.int64)
    rep_ids = np.asarray(rep_ids, dtype=np.int64)
    rcounts = np.diff(rep_off)
    off = np.zeros(nlist + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts + rcounts)
    ids = np.empty(off[-1], dtype=np.int64)
    pstart = np.zeros(nlist + 1, dtype=np.int64)
    pstart[1:] = np.cumsum(counts)
    for l in range(nlist):
        a = off[l]
        ids[a:a + counts[l]] = order[pstart[l]:pstart[l + 1]]
        ids[a + counts[l]:off[l + 1]] = rep_ids[rep_off[l]:rep_off[l + 1]]
    return off, ids


# ---------------------------------------------------------------------------
# step wrappers
# ---------------------------------------------------------------------------

def coarse(queries, centroids, nprobe, with_d2=False, metric=L2):
    q = _c(queries, np.float32)
    c = _c(centroids, np.float32)
    nq, d = q.shape
    nlist = c.shape[0]
    probes = np.empty((nq, nprobe), dtype=np.int32)
    d2 = np.empty((nq, nprobe), dtype=np.float64) if with_d2 else None
    lib().or_coarse_m(_p(q), nq, d, _p(c), nlist, nprobe, _p(probes), _p(d2), metric)
    return (probes, d2) if with_d2 else probes


def lut(query, codebooks, metric=L2):
    q = _c(query, np.float32).reshape(-1)
    cb = _c(codebooks, np.float32)
    M = cb.shape[0]
    out = np.empty((M, 256), dtype=np.float64)
    lib().or_lut_m(_p(q), q.shape[0], M, _p(cb), _p(out), metric)
    return out


def candidates(probes, list_off, list_ids):
    """(sorted distinct ids as uint32, gathered count)."""
    pr = _c(probes, np.int32).reshape(-1)
    off = _c(list_off, np.int64)
    ids = _c(list_ids, np.int64)
    cap = int(sum(off[l + 1] - off[l] for l in pr)) or 1
    out = np.empty(cap, dtype=np.uint32)
    g = C.c_int64(0)
    u = lib().or_candidates(_p(pr), pr.shape[0], _p(off), _p(ids), _p(out), cap, C.byref(g))
    assert u >= 0
    return out[:u].copy(), int(g.value)


def adc(lut_table, codes, ids):
    t = _c(lut_table, np.float64)
    cd = _c(codes, np.uint8)
    ii = _c(ids, np.uint32)
    out = np.empty(ii.shape[0], dtype=np.float64)
    lib().or_adc(_p(t), t.shape[0], _p(cd), _p(ii), ii.shape[0], _p(out))
    return out


def topn(dist, ids, n):
    dd = _c(dist, np.float64)
    ii = _c(ids, np.uint32)
    oi = np.empty(n, dtype=np.int64)
    od = np.empty(n, dtype=np.float64)
    lib().or_topn(_p(dd), _p(ii), dd.shape[0], n, _p(oi), _p(od))
    return oi, od


def exact(query, raw, ids, metric=L2):
    """Exact distances of the given rows: squared L2, or -<q, x> for IP."""
    q = _c(query, np.float32).reshape(-1)
    r = np.ascontiguousarray(raw)
    ii = _c(ids, np.int64)
    out = np.empty(ii.shape[0], dtype=np.float64)
    lib().or_exact_m(_p(q), q.shape[0], _p(r), raw_kind(r), _p(ii), ii.shape[0], _p(out), metric)
    return out


def exact_l2(query, raw, ids):
    return exact(query, raw, ids, L2)


def rerank(query, raw, tasks, k, batch=32, eps=0.0, beta=2, metric=L2):
    """Algorithm 1 on one query: (ids, exact dists, mini-batches run)."""
    q = _c(query, np.float32).reshape(-1)
    r = np.ascontiguousarray(raw)
    t = _c(tasks, np.int64)
    oi = np.empty(k, dtype=np.int64)
    od = np.empty(k, dtype=np.float64)
    nb = lib().or_rerank_m(_p(q), q.shape[0], _p(r), raw_kind(r), _p(t), t.shape[0], k, batch,
                           float(eps), beta, _p(oi), _p(od), metric)
    return oi, od, int(nb)


def search(queries, centroids, codebooks, codes, list_off, list_ids, nprobe, k, raw=None,
           probes=None, rerank_n=0, batch=32, eps=0.0, beta=2, stats=False, metric=L2):
    """The whole filtering path for every query: (ids [nq][k], dists, stats?)."""
    q = _c(queries, np.float32)
    nq, d = q.shape
    cent = _c(centroids, np.float32)
    cb = _c(codebooks, np.float32)
    cd = _c(codes, np.uint8)
    off = _c(list_off, np.int64)
    ids = _c(list_ids, np.int64)
    nlist, M = cent.shape[0], cb.shape[0]
    nprobe = max(1, min(int(nprobe), nlist))
    pr = None if probes is None else _c(probes, np.int32)
    r = None if raw is None else np.ascontiguousarray(raw)
    if rerank_n > 0 and r is None:
        raise ValueError("re-rank needs raw vectors")
    oi = np.empty((nq, k), dtype=np.int64)
    od = np.empty((nq, k), dtype=np.float64)
    st = np.empty((nq, 4), dtype=np.int64)
    rc = lib().or_search_m(_p(q), nq, d, _p(cent), nlist, M, _p(cb), _p(cd), _p(off), _p(ids),
                           _p(r), 0 if r is None else raw_kind(r), nprobe, k, _p(pr), rerank_n,
                           batch, float(eps), beta, _p(oi), _p(od), _p(st), metric)
    if rc != 0:
        raise RuntimeError("oracle search failed")
    return (oi, od, st) if stats else (oi, od)


def knn(queries, base, k, metric=L2):
    """Brute-force exact k-NN (FP64, ties by smaller id): (ids, dists)."""
    q = _c(queries, np.float32)
    b = np.ascontiguousarray(base)
    nq, d = q.shape
    oi = np.empty((nq, k), dtype=np.int64)
    od = np.empty((nq, k), dtype=np.float64)
    lib().or_knn_m(_p(q), nq, _p(b), raw_kind(b), b.shape[0], d, k, _p(oi), _p(od), metric)
    return oi, od


def recall_at(found_ids, gt_ids, gt_dist, exact_found_dist=None, at=10):
    """Recall@at: |found ∩ GT| / at per query, averaged (the paper's Recall@10,
    §6). Tie-aware when exact_found_dist is given: a returned id whose exact
    distance is <= the at-th ground-truth distance also counts."""
    f = np.asarray(found_ids)[:, :at]
    g = np.asarray(gt_ids)[:, :at]
    hits = np.zeros(f.shape[0])
    for i in range(f.shape[0]):
        gs = set(int(x) for x in g[i] if x >= 0)
        h = 0
        for t, x in enumerate(f[i]):
            if x < 0:
                continue
            if int(x) in gs:
                h += 1
            elif exact_found_dist is not None and exact_found_dist[i, t] <= gt_dist[i, at - 1]:
                h += 1
        hits[i] = min(h, at) / at
    return float(hits.mean())


def page_layout(primary, nlist, cap):
    """§4.3's storage layout: (page of each vector, slot in its page, pages)."""
    pr = _c(primary, np.int32)
    n = pr.shape[0]
    page_of = np.empty(n, dtype=np.int64)
    slot_of = np.empty(n, dtype=np.int32)
    np_ = lib().or_page_layout(_p(pr), n, nlist, cap, _p(page_of), _p(slot_of))
    return page_of, slot_of, int(np_)


def rerank_pages(query, raw, tasks, k, page_of, batch=32, eps=0.0, beta=2, metric=L2):
    """Algorithm 1 with §4.3's intra- and inter-mini-batch I/O deduplication:
    (ids, exact dists, mini-batches run, pages read)."""
    q = _c(query, np.float32).reshape(-1)
    r = np.ascontiguousarray(raw)
    t = _c(tasks, np.int64)
    pg = _c(page_of, np.int64)
    oi = np.empty(k, dtype=np.int64)
    od = np.empty(k, dtype=np.float64)
    reads = C.c_int64(0)
    nb = lib().or_rerank_pages(_p(q), q.shape[0], _p(r), raw_kind(r), _p(t), t.shape[0], k, batch,
                               float(eps), beta, _p(pg), _p(oi), _p(od), metric, C.byref(reads))
    return oi, od, int(nb), int(reads.value)



def graph_heads(centroids, raw_dtype):
    """The navigation graph's vertex vectors (§4.1): the centroids, rounded
    and clipped to the data's integer grid for uint8 / int8 vectors.
    raw_dtype: the numpy dtype of the raw vectors."""
    c = _c(centroids, np.float32)
    kind = {np.dtype(np.uint8): 1, np.dtype(np.int8): 2}.get(np.dtype(raw_dtype), 0)
    h = np.empty(c.shape, dtype=np.float64)
    lib().or_graph_heads(_p(c), c.shape[0], c.shape[1], kind, _p(h))
    return h


def graph_probe(queries, heads, adj, seeds, beam, max_check, nprobe, metric=L2):
    """Step 2 by the navigation graph (§3, §4.1): the best-first walk from the
    seeds with a beam of ``beam`` vertices and at most ``max_check`` checked
    vertices before an expansion. ``seeds``: one list for every query, or a
    [nq][S] array of each query's own seeds. Returns (lists [nq][nprobe], -1
    padded; lists found per query; vertices checked per query)."""
    q = _c(queries, np.float32)
    h = _c(heads, np.float64)
    a = _c(adj, np.int32)
    nq, d = q.shape
    sd = _c(seeds, np.int32)
    if sd.ndim == 2:
        assert sd.shape[0] == nq
        S, stride = sd.shape[1], sd.shape[1]
    else:
        S, stride = sd.shape[0], 0
    out = np.empty((nq, nprobe), dtype=np.int32)
    found = np.empty(nq, dtype=np.int32)
    checks = np.empty(nq, dtype=np.int32)
    lib().or_graph_probe(_p(q), nq, d, _p(h), h.shape[0], _p(a), a.shape[1], _p(sd), S, stride, beam,
                         max_check, nprobe, metric, _p(out), _p(found), _p(checks))
    return out, found, checks


def graph_entry(queries, heads, pivots, entry, metric=L2):
    """Each query's own seeds: the ``entry`` pivot vertices nearest to it
    (the exact top-entry probe of the pivots' heads, ties by pivot order),
    as vertex ids [nq][entry]."""
    pv = _c(pivots, np.int32)
    near = coarse(queries, np.asarray(heads, np.float64)[pv].astype(np.float32), entry, metric=metric)
    return pv[near]
