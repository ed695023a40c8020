"""Parity of the batched form (FA_BATCHED: the whole batch scanned list by
list, two queries' FP16 entries per shared-memory table word) with the FP64
oracle, through the C ABI.

The batched form's distances come from an FP16 table with one scale per
query, so each is checked against the oracle's FP64 ADC of the same id within
the table's error bound, and the top-n against the oracle's within that
bound. Gather and dedup are checked exactly: with k above a query's candidate
count every distinct candidate comes back, and the set equals the oracle's
sort-unique of the probed lists (replication on). The exhaustive re-rank is
checked bit for bit against the oracle's Algorithm 1 on the GPU's own top-n.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_checks import (_adc_ref, _batched_adc_bound, _batched_entry_bound, _check_bounded_topn,
                           _l2_ref)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_16576_b300 as m
    return m


def _lists(parts):
    return oracle.lists_from_parts(parts["primary"], parts["rep_off"], parts["rep_ids"], parts["nlist"])


def _bp(fa, tc=True, prec="F16", **kw):
    g = fa.FA_GEMM_BF16_TC if tc else fa.FA_GEMM_SIMT_F32
    flags = fa.FA_BATCHED | kw.pop("flags", 0)
    return fa.search_params(lut_prec=getattr(fa, "FA_LUT_" + prec), lut_gemm=g, probe_gemm=g, flags=flags,
                            **kw)


@pytest.fixture(scope="module")
def u8_repl(fa):
    """uint8 d=128 vectors with Eq. 2 replication (up to 4 lists per vector)."""
    mix = synth.Mixture(128, 16, 8.0, kind="u8")
    base = mix.base(30_000)
    q = mix.queries(40)
    ix = fa.fa_build_index(base, fa.build_params(nlist=64, M=32, kmeans_iters=6, repl_eps=0.08,
                                                 max_lists_per_vec=4,
                                                 raw_location=fa.FA_RAW_HOST_PINNED))
    parts = ix.parts()
    assert parts["rep_off"][-1] > 0
    off, ids = _lists(parts)
    return dict(base=base, q=q, ix=ix, parts=parts, off=off, ids=ids)


@pytest.fixture(scope="module")
def u8_dev(fa):
    """uint8 d=128 vectors, raw rows in HBM (the fused exhaustive re-rank)."""
    mix = synth.Mixture(128, 16, 8.0, kind="u8")
    base = mix.base(40_000)
    q = mix.queries(24)
    ix = fa.fa_build_index(base, fa.build_params(nlist=64, M=32, kmeans_iters=6,
                                                 raw_location=fa.FA_RAW_DEVICE))
    parts = ix.parts()
    off, ids = _lists(parts)
    return dict(base=base, q=q, ix=ix, parts=parts, off=off, ids=ids)


@pytest.fixture(scope="module")
def f32_small(fa):
    w = synth.plain_f32_100k()
    base = w.mix.base(w.n)
    q = w.mix.queries(w.nq)
    ix = fa.fa_build_index(base, fa.build_params(nlist=w.nlist, M=w.M, kmeans_iters=8,
                                                 raw_location=fa.FA_RAW_DEVICE))
    parts = ix.parts()
    off, ids = _lists(parts)
    return dict(base=base, q=q, ix=ix, parts=parts, off=off, ids=ids)


def _bounded(fa, s, q, k, npb, params, probes, tc=True, what="", prec="F16"):
    gi, gd = fa.fa_search_ex(s["ix"], q, k, npb, params, probes=probes)
    oi, _ = oracle.search(q, s["parts"]["centroids"], s["parts"]["codebooks"], s["parts"]["codes"],
                          s["off"], s["ids"], npb, k, probes=probes)
    for i in range(q.shape[0]):
        _check_bounded_topn(gi[i], gd[i], oi[i], _adc_ref(q[i], s["parts"]),
                            _batched_adc_bound(q[i], s["parts"], tc, prec), what="%s q%d" % (what, i))
    return gi, gd


@pytest.mark.parametrize("k", [1, 10, 100, 600, 3000])
@pytest.mark.parametrize("tc", [True, False])
@pytest.mark.parametrize("prec", ["F16", "FP8"])
def test_batched_topk_with_replication(fa, u8_repl, k, tc, prec):
    """Replicated lists (dedup at work), top-n from the warp and CTA sizes,
    FP16 pairs and FP8 quadruples of queries per table word: every distance
    within the table's bound of the oracle's ADC, and the top-n the
    oracle's within that bound."""
    s = u8_repl
    probes = oracle.coarse(s["q"], s["parts"]["centroids"], 16)
    _bounded(fa, s, s["q"], k, 16, _bp(fa, tc, prec), probes, tc, what="k%d" % k, prec=prec)


@pytest.mark.parametrize("prec", ["F16", "FP8"])
def test_batched_gather_and_dedup_exact(fa, u8_repl, prec):
    """k above every query's candidate count: the returned ids are exactly the
    oracle's distinct candidates of the probed lists (bit-exact gather and
    dedup over replicated lists), and the statistics count them."""
    s = u8_repl
    q = s["q"][:12]
    rng = np.random.default_rng(8)
    nl = s["parts"]["nlist"]
    probes = np.stack([rng.choice(nl, size=10, replace=False) for _ in range(q.shape[0])]).astype(np.int32)
    gi, gd, st = fa.fa_search_ex(s["ix"], q, 16384, 10, _bp(fa, prec=prec), probes=probes, stats=True)
    for i in range(q.shape[0]):
        ref, gathered = oracle.candidates(probes[i], s["off"], s["ids"])
        got = gi[i][gi[i] >= 0]
        assert sorted(got.tolist()) == ref.astype(np.int64).tolist(), i
        assert st[i, 0] == gathered and st[i, 1] == ref.shape[0], (i, st[i])


@pytest.mark.parametrize("shift,sigma", [(0.0, 4.0), (0.3, 4.0), (0.0, -1000.0)])
@pytest.mark.parametrize("n", [1000, 3000])
def test_batched_fused_rerank_matches_oracle(fa, u8_dev, n, shift, sigma):
    """Exhaustive Algorithm 1 (eps < 0) fused after the batched selection:
    the oracle's Algorithm 1 on the GPU's own batched ADC top-n gives the
    GPU's ids and distances (bit for bit for integral queries). Sigma -1000
    puts every threshold too low, so every query takes the redo path."""
    s = u8_dev
    k, npb = 10, 24
    q = (s["q"] + np.float32(shift)).astype(np.float32)
    probes = oracle.coarse(q, s["parts"]["centroids"], npb)
    fa.fa_debug_tau_sigma(sigma)
    try:
        gi, gd, st = fa.fa_search_ex(s["ix"], q, k, npb, _bp(fa, rerank_n=n, rerank_eps=-1.0),
                                     probes=probes, stats=True)
        an_i, an_d = _bounded(fa, s, q, n, npb, _bp(fa), probes, what="adc")
    finally:
        fa.fa_debug_tau_sigma(4.0)
    for i in range(q.shape[0]):
        tasks = an_i[i][an_i[i] >= 0]
        oi, od, nb = oracle.rerank(q[i], s["parts"]["raw"], tasks, k, batch=32, eps=-1.0, beta=1)
        if shift == 0.0:
            assert gd[i].tolist() == od.astype(np.float32).tolist(), i
            assert gi[i].tolist() == oi.tolist(), i
        else:
            np.testing.assert_allclose(gd[i], _l2_ref(q[i], s["parts"]["raw"])(gi[i]), rtol=1e-5)
            assert set(gi[i].tolist()) == set(oi.tolist()) or np.isclose(od[-1], gd[i][-1], rtol=1e-5)
        assert st[i, 3] == len(tasks), (i, st[i])


@pytest.mark.parametrize("k,sigma", [(4097, -1000.0), (4097, 4.0), (4097, 150.0), (600, 400.0)])
def test_batched_every_threshold_path(fa, f32_small, k, sigma):
    """100k candidates per query (every one of the 256 lists probed), more
    than a query's key buffer holds (65536 keys): the sampled threshold
    filters. Forced low (fewer than n keys below it) or high (more keys than
    the buffer holds), the queries are handed to the per-query scan; all
    paths meet the bound."""
    s = f32_small
    q = s["q"][:8]
    npb = s["parts"]["nlist"]
    probes = oracle.coarse(q, s["parts"]["centroids"], npb)
    fa.fa_debug_tau_sigma(sigma)
    try:
        _bounded(fa, s, q, k, npb, _bp(fa), probes, what="sigma%g" % sigma)
    finally:
        fa.fa_debug_tau_sigma(4.0)


def test_batched_per_query_k_and_nprobe(fa, f32_small):
    s = f32_small
    q = s["q"][:30]
    rng = np.random.default_rng(19)
    kq = rng.integers(1, 11, size=30).astype(np.int32)
    npq = rng.integers(1, 9, size=30).astype(np.int32)
    probes = oracle.coarse(q, s["parts"]["centroids"], 8)
    gi, gd = fa.fa_search_ex(s["ix"], q, 10, 8, _bp(fa), probes=probes, k_per_query=kq,
                             nprobe_per_query=npq)
    for i in range(30):
        oi, _ = oracle.search(q[i:i + 1], s["parts"]["centroids"], s["parts"]["codebooks"],
                              s["parts"]["codes"], s["off"], s["ids"], int(npq[i]), int(kq[i]),
                              probes=probes[i:i + 1, :npq[i]])
        _check_bounded_topn(gi[i, :kq[i]], gd[i, :kq[i]], oi[0], _adc_ref(q[i], s["parts"]),
                            _batched_adc_bound(q[i], s["parts"], True), what=str(i))
        assert np.all(gi[i, kq[i]:] == -1) and np.all(np.isinf(gd[i, kq[i]:]))


@pytest.mark.parametrize("prec", ["F16", "FP8"])
def test_batched_uneven_lists_in_tiles(fa, prec):
    """Zipf(1.1) list sizes (the largest list spans two 1024-chunk tiles):
    the batched form over per-query nprobe meets the bound."""
    rng = np.random.default_rng(33)
    n, d, M, nlist = 150_000, 32, 16, 64
    sizes = synth.zipf_sizes(nlist, n)
    primary = np.repeat(np.arange(nlist, dtype=np.int32), sizes)
    rng.shuffle(primary)
    cent = rng.normal(size=(nlist, d)).astype(np.float32)
    cb = rng.normal(size=(M, 256, d // M)).astype(np.float32)
    codes = rng.integers(0, 256, size=(n, M)).astype(np.uint8)
    ix = fa.fa_index_from_parts(cent, cb, codes, primary)
    parts = ix.parts()
    off, ids = _lists(parts)
    s = dict(ix=ix, parts=parts, off=off, ids=ids)
    assert sizes.max() > 1024 * 32  # at least two tiles
    q = rng.normal(size=(50, d)).astype(np.float32)
    npq = rng.integers(1, 17, size=50).astype(np.int32)
    probes = oracle.coarse(q, cent, 16)
    for k in (10, 100):
        gi, gd = fa.fa_search_ex(ix, q, k, 16, _bp(fa, prec=prec), probes=probes, nprobe_per_query=npq)
        for i in range(50):
            oi, _ = oracle.search(q[i:i + 1], cent, parts["codebooks"], parts["codes"], off, ids,
                                  int(npq[i]), k, probes=probes[i:i + 1, :npq[i]])
            _check_bounded_topn(gi[i], gd[i], oi[0], _adc_ref(q[i], parts),
                                _batched_adc_bound(q[i], parts, True, prec), what="k%d q%d" % (k, i))


def test_batched_sorted_rows_for_early_stop(fa, u8_repl):
    """Algorithm 1 with early stopping (eps 0, beta 2) reads the top-n in ADC
    order: the batched selection sorts its rows, and the oracle's Algorithm 1
    on the GPU's batched ADC top-50 gives the GPU's result bit for bit."""
    s = u8_repl
    q = s["q"][:20]
    probes = oracle.coarse(q, s["parts"]["centroids"], 16)
    gi, gd, st = fa.fa_search_ex(s["ix"], q, 10, 16, _bp(fa, rerank_n=50, rerank_eps=0.0, rerank_beta=2),
                                 probes=probes, stats=True)
    an_i, an_d = _bounded(fa, s, q, 50, 16, _bp(fa), probes)
    compared = 0
    for i in range(q.shape[0]):
        tasks = an_i[i][an_i[i] >= 0]
        if len(np.unique(an_d[i][:len(tasks)])) != len(tasks):
            continue  # equal ADC keys: the order among them is the GPU's
        oi, od, nb = oracle.rerank(q[i], s["parts"]["raw"], tasks, 10, batch=32, eps=0.0, beta=2)
        assert gi[i].tolist() == oi.tolist(), i
        assert gd[i].tolist() == od.astype(np.float32).tolist(), i
        assert st[i, 2] == nb, (i, st[i], nb)
        compared += 1
    assert compared >= q.shape[0] // 2


def test_batched_graph_capture_replays(fa, u8_repl):
    """FA_GRAPH with FA_BATCHED: the captured search replays and reads new
    query contents in the same buffer; it equals the uncaptured call."""
    import torch
    s = u8_repl
    qd = torch.as_tensor(s["q"], device="cuda")
    oi = torch.empty((qd.shape[0], 10), dtype=torch.int64, device="cuda")
    od = torch.empty((qd.shape[0], 10), dtype=torch.float32, device="cuda")
    for rnd in range(3):
        if rnd == 2:
            qd.copy_(torch.flip(qd, [0]))
        fa.fa_search_ex(s["ix"], qd, 10, 12, _bp(fa, flags=fa.FA_GRAPH), out_ids=oi, out_dist=od)
        torch.cuda.synchronize()
        ei, ed = fa.fa_search_ex(s["ix"], qd.cpu().numpy(), 10, 12, _bp(fa))
        assert np.array_equal(oi.cpu().numpy(), ei), rnd
        assert np.array_equal(od.cpu().numpy().view(np.uint32), ed.view(np.uint32)), rnd


@pytest.mark.parametrize("prec", ["F16", "FP8"])
def test_batched_lut_has_one_scale_per_query(fa, u8_repl, prec):
    """The table the batched form reads (fa_debug_lut with FA_BATCHED): one
    scale per query; each entry within the bound the tests above use."""
    s = u8_repl
    for tc in (True, False):
        p = _bp(fa, tc, prec)
        for i in range(3):
            got = fa.fa_debug_lut(s["ix"], s["q"][i], p).astype(np.float64)
            ref, _, bound = _batched_entry_bound(s["q"][i], s["parts"], tc, prec)
            assert np.all(np.abs(got - ref) <= bound), (tc, i, float(np.max(np.abs(got - ref) - bound)))
