"""Coarse probe by the navigation graph (§3 step 2, §4.1 "In-memory Indices").

The graph is part of the index (an input to both sides, like the lists): it
is exported and the oracle walks it. Checked against the oracle:
  * the build: every vertex's out-edges follow the build's rule (pruned
    nearest heads, reverse edges, nearest fill) computed from the oracle's
    exact probe of the heads against themselves, and the heads are the
    oracle's rounding of the centroids;
  * the walk: for integer vectors with integral queries every distance is an
    integer (exact in FP32), so the GPU's walk takes the oracle's FP64
    decisions: the entry pivots, lists, lists found and vertices checked are
    equal for every query, over beams of 1..256 (every register width of the
    beam), small and large check budgets, walks from every pivot and from the
    nearest few, uint8 and int8 vectors, L2 and inner product;
  * float vectors: FP32 rounding may flip a near tie, so most walks must
    equal the oracle's and every walk must return distinct lists in the
    oracle's distance order;
  * the search: FA_PROBE_GRAPH returns what a search over the oracle's walk
    lists returns (the scan after the probe is the scan of those lists),
    with the table built on the second stream.
"""
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
    if "u8" not in _CACHE:
        mix = synth.Mixture(128, 256, 8.0, kind="u8")
        base = mix.base(150_000)
        q = mix.queries(200)
        ix = fa.fa_build_index(base, fa.build_params(nlist=2048, M=32, kmeans_iters=4,
                                                     raw_location=fa.FA_RAW_DEVICE))
        fa.fa_build_probe_graph(ix, 24, 40)
        parts = ix.parts()
        g = fa.fa_index_get_graph(ix)
        heads = oracle.graph_heads(parts["centroids"], np.uint8)
        _CACHE["u8"] = dict(base=base, q=q, ix=ix, parts=parts, g=g, heads=heads, metric=oracle.L2)
    return _CACHE["u8"]


def _i8(fa, metric):
    key = "i8" + metric
    if key not in _CACHE:
        mix = synth.spacev_like(1_000_000, 25).mix
        base = mix.base(60_000)
        q = mix.queries(120)
        ix = fa.fa_build_index(base, fa.build_params(nlist=1024, M=25, kmeans_iters=4,
                                                     metric=getattr(fa, "FA_METRIC_" + metric)))
        fa.fa_build_probe_graph(ix, 16, 32)
        parts = ix.parts()
        g = fa.fa_index_get_graph(ix)
        heads = oracle.graph_heads(parts["centroids"], np.int8)
        _CACHE[key] = dict(q=q, ix=ix, parts=parts, g=g, heads=heads,
                           metric=oracle.IP if metric == "IP" else oracle.L2)
    return _CACHE[key]


def test_graph_edges_follow_the_build_rule(fa):
    """Out-edges of every vertex by the build's rule, from the oracle's exact
    K = 3R nearest heads (distance, id) and FP64 distances between heads:
    relative-neighbourhood pruning, then the vertices that kept it (nearest
    first), then its nearest candidates."""
    s = _u8(fa)
    g, heads = s["g"], s["heads"]
    R = g["R"]
    assert R == 24 and g["S"] == 40
    h32 = heads.astype(np.float32)
    nlist, K = heads.shape[0], 3 * R
    nn = oracle.coarse(h32, h32, K + 1)

    def hd(a, b):
        return float(((heads[a] - heads[b]) ** 2).sum())
    first = []
    for p in range(nlist):
        kept = []
        for c in nn[p].tolist():
            if c == p or len(kept) >= R:
                continue
            dpc = hd(p, c)
            if all(hd(n, c) >= dpc for n in kept):
                kept.append(c)
        first.append(kept)
    rev = [[] for _ in range(nlist)]
    for v in range(nlist):
        for u in first[v]:
            rev[u].append((hd(u, v), v))
    for u in range(nlist):
        want = []
        for x in first[u] + [w for _, w in sorted(rev[u])] + nn[u].tolist():
            if x != u and x not in want and len(want) < R:
                want.append(x)
        assert g["adj"][u].tolist() == want + [-1] * (R - len(want)), u
    nlist = heads.shape[0]
    assert g["seeds"].tolist() == [i * nlist // 40 for i in range(40)]


def _seeds(s, entry, metric=oracle.L2):
    """The oracle's seeds of each walk: every pivot, or the entry nearest."""
    g = s["g"]
    if entry >= g["S"]:
        return g["seeds"]
    return oracle.graph_entry(s["q"], s["heads"], g["seeds"], entry, metric=metric)


@pytest.mark.parametrize("entry", [40, 5])
@pytest.mark.parametrize("beam,max_check,nprobe", [(1, 400, 1), (32, 200, 16), (48, 20, 48), (100, 600, 64),
                                                   (256, 3000, 200), (64, 0, 32)])
def test_graph_walk_equals_oracle_u8(fa, beam, max_check, nprobe, entry):
    s = _u8(fa)
    g = s["g"]
    got, found, checks = fa.fa_debug_graph_probe(s["ix"], s["q"], nprobe, beam, max_check, entry)
    mc = max_check if max_check > 0 else 16 * nprobe + min(entry, g["S"])  # the library's default budget
    ref, rfound, rchecks = oracle.graph_probe(s["q"], s["heads"], g["adj"], _seeds(s, entry), beam, mc, nprobe)
    assert np.array_equal(found, rfound)
    assert np.array_equal(checks, rchecks)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("metric", ["L2", "IP"])
def test_graph_walk_equals_oracle_i8(fa, metric):
    s = _i8(fa, metric)
    g = s["g"]
    for beam, mc, nprobe, entry in ((64, 500, 32, 32), (128, 60, 128, 32), (64, 500, 32, 6)):
        got, found, checks = fa.fa_debug_graph_probe(s["ix"], s["q"], nprobe, beam, mc, entry)
        ref, rfound, rchecks = oracle.graph_probe(s["q"], s["heads"], g["adj"], _seeds(s, entry, s["metric"]),
                                                  beam, mc, nprobe, metric=s["metric"])
        assert np.array_equal(found, rfound) and np.array_equal(checks, rchecks)
        assert np.array_equal(got, ref)


def test_graph_walk_float_vectors(fa):
    """Float heads (the centroids): FP32 rounding may flip a near tie."""
    mix = synth.Mixture(64, 64, 8.0)
    base = mix.base(40_000)
    q = mix.queries(150)
    ix = fa.fa_build_index(base, fa.build_params(nlist=512, M=16, kmeans_iters=4))
    fa.fa_build_probe_graph(ix, 16, 16)
    parts = ix.parts()
    g = fa.fa_index_get_graph(ix)
    heads = oracle.graph_heads(parts["centroids"], np.float32)
    nprobe, beam, mc = 24, 48, 400
    got, found, checks = fa.fa_debug_graph_probe(ix, q, nprobe, beam, mc, 16)
    ref, rfound, _ = oracle.graph_probe(q, heads, g["adj"], g["seeds"], beam, mc, nprobe)
    same = np.all(got == ref, axis=1)
    assert same.mean() >= 0.95, same.mean()
    assert np.all(found == nprobe) and np.all(rfound == nprobe)
    for i in range(q.shape[0]):
        row = got[i]
        assert len(set(row.tolist())) == nprobe, i
        d2 = ((heads[row] - q[i].astype(np.float64)) ** 2).sum(axis=1)
        assert np.all(np.diff(d2) >= -1e-5 * np.maximum(d2[1:], 1.0)), i


@pytest.mark.parametrize("prec", ["F32", "F16"])
def test_search_with_graph_probe_equals_search_of_walk_lists(fa, prec):
    """FA_PROBE_GRAPH (the table on the second stream in the FP16 form) equals
    a search given the oracle's walk lists, with per-query list counts."""
    s = _u8(fa)
    g = s["g"]
    nprobe, beam, mc = 32, 64, 600
    tc = fa.FA_GEMM_BF16_TC
    base = dict(lut_prec=getattr(fa, "FA_LUT_" + prec), lut_gemm=tc if prec == "F16" else fa.FA_GEMM_SIMT_F32,
                rerank_n=200, rerank_eps=-1.0, rerank_beta=1)
    p = fa.search_params(probe_gemm=fa.FA_PROBE_GRAPH, graph_beam=beam, graph_max_check=mc, **base)
    gi, gd = fa.fa_search_ex(s["ix"], s["q"], 10, nprobe, p)
    # the default entry: the 16 pivots nearest each query
    ref, rfound, _ = oracle.graph_probe(s["q"], s["heads"], g["adj"], _seeds(s, 16), beam, mc, nprobe)
    pr = np.where(ref < 0, 0, ref).astype(np.int32)
    ri, rd = fa.fa_search_ex(s["ix"], s["q"], 10, nprobe, fa.search_params(**base), probes=pr,
                             nprobe_per_query=rfound)
    assert np.array_equal(gi, ri) and np.array_equal(gd, rd)


def test_graph_probe_finds_most_exact_lists(fa):
    """The walk's lists against the exact top-m with the default graph and
    budget: most of them (0.94 measured; a quality check of the graph, not a parity
    check; on this mixture a graph of 24 edges and 40 seeds finds ~0.73)."""
    s = _u8(fa)
    nprobe = 32
    fa.fa_build_probe_graph(s["ix"])
    try:
        got, found, _ = fa.fa_debug_graph_probe(s["ix"], s["q"], nprobe)
        exact = oracle.coarse(s["q"], s["parts"]["centroids"], nprobe)
        hit = np.mean([len(set(got[i, :found[i]].tolist()) & set(exact[i].tolist())) / nprobe
                       for i in range(s["q"].shape[0])])
        assert hit >= 0.9, hit
    finally:
        fa.fa_build_probe_graph(s["ix"], 24, 40)  # the graph the other tests exported


def test_graph_probe_arguments(fa):
    s = _u8(fa)
    with pytest.raises(fa.FaError) as e:  # beam below nprobe
        fa.fa_debug_graph_probe(s["ix"], s["q"][:2], 32, 16, 100)
    assert e.value.status == fa.FA_ERR_ARG
    with pytest.raises(fa.FaError) as e:
        fa.fa_build_probe_graph(s["ix"], 65, 8)
    assert e.value.status == fa.FA_ERR_ARG
    mix = synth.Mixture(32, 4, 8.0)
    ix = fa.fa_build_index(mix.base(2000), fa.build_params(nlist=16, M=8, kmeans_iters=2))
    with pytest.raises(fa.FaError) as e:  # no graph built
        fa.fa_search_ex(ix, mix.queries(2), 5, 4, fa.search_params(probe_gemm=fa.FA_PROBE_GRAPH))
    assert e.value.status == fa.FA_ERR_ARG


def test_batched_search_with_graph_probe(fa):
    """The batched form (FA_BATCHED, FP8 table) after the graph walk equals
    the batched form given the oracle's walk lists."""
    s = _u8(fa)
    g = s["g"]
    nprobe, beam, mc = 32, 64, 600
    tc = fa.FA_GEMM_BF16_TC
    base = dict(lut_prec=fa.FA_LUT_FP8, lut_gemm=tc, rerank_n=200, rerank_eps=-1.0, rerank_beta=1,
                flags=fa.FA_BATCHED)
    p = fa.search_params(probe_gemm=fa.FA_PROBE_GRAPH, graph_beam=beam, graph_max_check=mc, **base)
    gi, gd = fa.fa_search_ex(s["ix"], s["q"], 10, nprobe, p)
    ref, rfound, _ = oracle.graph_probe(s["q"], s["heads"], g["adj"], _seeds(s, 16), beam, mc, nprobe)
    pr = np.where(ref < 0, 0, ref).astype(np.int32)
    ri, rd = fa.fa_search_ex(s["ix"], s["q"], 10, nprobe, fa.search_params(**base), probes=pr,
                             nprobe_per_query=rfound)
    assert np.array_equal(gi, ri) and np.array_equal(gd, rd)


@pytest.mark.parametrize("nlist", [1, 2, 5])
def test_graph_probe_tiny_indexes(fa, nlist):
    """A graph of one, two or five lists (every walk reaches them all):
    FA_PROBE_GRAPH probing every list equals the exact probe of every list."""
    mix = synth.Mixture(32, 4, 8.0, kind="u8")
    base = mix.base(3000)
    q = mix.queries(20)
    ix = fa.fa_build_index(base, fa.build_params(nlist=nlist, M=8, kmeans_iters=3))
    fa.fa_build_probe_graph(ix)
    g = fa.fa_index_get_graph(ix)
    assert g["adj"].shape == (nlist, max(1, min(32, nlist - 1)))
    a = fa.fa_search_ex(ix, q, 10, nlist, fa.search_params(probe_gemm=fa.FA_PROBE_GRAPH))
    b = fa.fa_search_ex(ix, q, 10, nlist)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_graph_probe_under_graph_capture(fa):
    """FA_GRAPH with FA_PROBE_GRAPH: the captured search (the walk on the
    call's stream, the table on the second stream, joined before the scan)
    replays to the eager result, also after the queries' contents change."""
    import torch
    s = _u8(fa)
    tc = fa.FA_GEMM_BF16_TC
    kw = dict(lut_prec=fa.FA_LUT_F16, lut_gemm=tc, probe_gemm=fa.FA_PROBE_GRAPH, graph_beam=64,
              graph_max_check=600)
    p = fa.search_params(flags=fa.FA_GRAPH, **kw)
    ref = fa.search_params(**kw)
    qd = torch.as_tensor(s["q"], device="cuda")
    oi = torch.empty((qd.shape[0], 10), dtype=torch.int64, device="cuda")
    od = torch.empty((qd.shape[0], 10), dtype=torch.float32, device="cuda")
    for rnd in range(3):
        if rnd == 2:
            qd.copy_(torch.flip(qd, [0]))  # new contents in the same buffer
        fa.fa_search_ex(s["ix"], qd, 10, 32, p, out_ids=oi, out_dist=od)
        torch.cuda.synchronize()
        ei, ed = fa.fa_search_ex(s["ix"], qd.cpu().numpy(), 10, 32, ref)
        assert np.array_equal(oi.cpu().numpy(), ei) and np.array_equal(od.cpu().numpy(), ed), rnd


def test_graph_is_not_saved(fa, tmp_path):
    """The graph is not part of a saved index: a loaded index refuses
    FA_PROBE_GRAPH until its graph is built again, then walks as before."""
    s = _u8(fa)
    path = str(tmp_path / "g.idx")
    fa.fa_save_index(s["ix"], path)
    ix2 = fa.fa_load_index(path)
    with pytest.raises(fa.FaError) as e:
        fa.fa_debug_graph_probe(ix2, s["q"], 16, 32, 200, 40)
    assert e.value.status == fa.FA_ERR_ARG
    fa.fa_build_probe_graph(ix2, 24, 40)
    a = fa.fa_debug_graph_probe(ix2, s["q"], 16, 32, 200, 40)
    b = fa.fa_debug_graph_probe(s["ix"], s["q"], 16, 32, 200, 40)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
