"""Re-rank from the paged storage of §4.3 (FA_RAW_HOST_PAGED).

The raw vectors sit in 4 KB pages in pinned host memory, one bucket of whole
pages per list with the unaligned tails packed by the max-min rule, and the
re-rank reads whole pages: a page that several vectors of a mini-batch share
is read once (intra-mini-batch deduplication) and a page an earlier
mini-batch of the same query read is taken from the query's page buffer in
HBM (inter-mini-batch deduplication).

Checked against the oracle, never against the GPU itself: the layout the
index builds equals the oracle's page_layout bit for bit; each query's
re-rank returns the ids, exact distances and mini-batch count of the
oracle's Algorithm 1 on the GPU's own ADC top-n, and reads exactly as many
pages as the oracle's deduplication does on those tasks."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

_CACHE = {}


@pytest.fixture(scope="module")
def fa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_16576_b300 as m
    return m


def _u8(fa):
    """uint8 d=128 vectors (128-byte rows, 32 to a page) with Eq. 2
    replication, so a query's tasks include replicas."""
    if "u8" not in _CACHE:
        mix = synth.Mixture(128, 16, 8.0, kind="u8")
        base = mix.base(30_000)
        q = mix.queries(32)
        ix = fa.fa_build_index(base, fa.build_params(nlist=64, M=32, kmeans_iters=6, repl_eps=0.08,
                                                     max_lists_per_vec=4,
                                                     raw_location=fa.FA_RAW_HOST_PAGED))
        parts = ix.parts()
        assert parts["rep_off"][-1] > 0
        _CACHE["u8"] = dict(q=q, ix=ix, parts=parts, metric=oracle.L2)
    return _CACHE["u8"]


def _i8(fa, metric):
    """int8 d=100 vectors (100-byte rows, 40 to a page), M 25."""
    key = "i8" + metric
    if key not in _CACHE:
        mix = synth.spacev_like(1_000_000, 25).mix
        base = mix.base(20_000)
        q = mix.queries(24)
        ix = fa.fa_build_index(base, fa.build_params(nlist=48, M=25, kmeans_iters=6,
                                                     raw_location=fa.FA_RAW_HOST_PAGED,
                                                     metric=getattr(fa, "FA_METRIC_" + metric)))
        _CACHE[key] = dict(q=q, ix=ix, parts=ix.parts(), metric=oracle.IP if metric == "IP" else oracle.L2)
    return _CACHE[key]


@pytest.mark.parametrize("which", ["u8", "i8L2"])
def test_page_map_equals_oracle_layout(fa, which):
    s = _u8(fa) if which == "u8" else _i8(fa, "L2")
    pm = fa.fa_debug_page_map(s["ix"])
    rowb = s["parts"]["raw"].shape[1] * s["parts"]["raw"].itemsize
    assert pm["rows_per_page"] == 4096 // rowb
    po, so, npg = oracle.page_layout(s["parts"]["primary"], s["parts"]["nlist"], pm["rows_per_page"])
    assert pm["pages"] == npg
    assert np.array_equal(pm["page_of"], po)
    assert np.array_equal(pm["slot_of"], so)


def _check_paged(fa, s, k, n, eps, beta, batch, npb=12):
    q = s["q"]
    probes = oracle.coarse(q, s["parts"]["centroids"], npb, metric=s["metric"])
    p = fa.search_params(rerank_n=n, rerank_batch=batch, rerank_beta=beta, rerank_eps=eps)
    reads = np.full(q.shape[0], -1, np.int32)
    gi, gd, st = fa.fa_search_ex(s["ix"], q, k, npb, p, probes=probes, stats=True, page_reads=reads)
    an_i, an_d = fa.fa_search_ex(s["ix"], q, n, npb, probes=probes)
    page_of = fa.fa_debug_page_map(s["ix"])["page_of"]
    compared = 0
    for i in range(q.shape[0]):
        tasks = an_i[i][an_i[i] >= 0]
        # with early stopping the mini-batches follow the ADC order, which an
        # ADC tie leaves to the id order of the internal layout: skip a query
        # whose tie straddles a mini-batch boundary
        cut = np.arange(batch, len(tasks), batch)
        if eps >= 0 and np.any(an_d[i][cut - 1] == an_d[i][cut]):
            continue
        oi, od, nb, rd = oracle.rerank_pages(q[i], s["parts"]["raw"], tasks, k, page_of, batch=batch,
                                             eps=eps, beta=beta, metric=s["metric"])
        assert gi[i].tolist() == oi.tolist(), (eps, i)
        assert gd[i].tolist() == od.astype(np.float32).tolist(), (eps, i)
        assert st[i, 2] == nb, (eps, i, st[i], nb)
        assert reads[i] == rd, (eps, i, reads[i], rd)
        # deduplication: never more pages than tasks re-ranked, never fewer
        # than the distinct pages of the first mini-batch
        assert len(np.unique(page_of[tasks[:batch]])) <= rd <= min(len(tasks), nb * batch)
        compared += 1
    assert compared >= q.shape[0] // 2
    return gi, gd


@pytest.mark.parametrize("eps,beta,batch,n", [(0.0, 2, 32, 300), (-1.0, 1, 32, 600), (0.1, 1, 64, 1000),
                                              (0.0, 3, 96, 4096)])
def test_paged_rerank_matches_oracle_pages(fa, eps, beta, batch, n):
    """uint8 rows, Algorithm 1 with and without early stopping, mini-batches
    of one, two and three warp steps, top-n up to 4096 (a buffer of 4096
    pages a warp)."""
    _check_paged(fa, _u8(fa), 10, n, eps, beta, batch)


@pytest.mark.parametrize("metric", ["L2", "IP"])
def test_paged_rerank_int8_matches_oracle_pages(fa, metric):
    """int8 rows of 100 bytes (pages of 40 rows, 4000 bytes), both metrics."""
    s = _i8(fa, metric)
    for eps, beta in ((-1.0, 1), (0.0, 2)):
        _check_paged(fa, s, 10, 400, eps, beta, 32)


def test_paged_rerank_equals_rows_in_hbm(fa):
    """The same index with its raw vectors in HBM returns the same ids and
    distances: paging changes what is read, not the result."""
    s = _u8(fa)
    pr = s["parts"]
    dev = fa.fa_index_from_parts(pr["centroids"], pr["codebooks"], pr["codes"], pr["primary"],
                                 pr["rep_off"], pr["rep_ids"], raw=pr["raw"],
                                 raw_location=fa.FA_RAW_DEVICE)
    probes = oracle.coarse(s["q"], pr["centroids"], 12)
    for eps, beta in ((-1.0, 1), (0.0, 2)):
        p = fa.search_params(rerank_n=500, rerank_eps=eps, rerank_beta=beta)
        a = fa.fa_search_ex(s["ix"], s["q"], 10, 12, p, probes=probes)
        b = fa.fa_search_ex(dev, s["q"], 10, 12, p, probes=probes)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), eps


def test_paged_rerank_rejects_page_reads_without_pages(fa):
    s = _u8(fa)
    reads = np.zeros(s["q"].shape[0], np.int32)
    with pytest.raises(fa.FaError) as e:  # no re-rank: no pages are read
        fa.fa_search_ex(s["ix"], s["q"], 10, 12, page_reads=reads)
    assert e.value.status == fa.FA_ERR_ARG
