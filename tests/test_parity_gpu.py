"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars (FP32 form): gather + dedup bit-exact; distances within 1e-4 relative;
top-k id sets equal except where the oracle's distances at the k boundary are
closer than that tolerance (several answers are then correct; the test checks
that the returned ones are valid). Inputs are seeded synthetic data shaped
like the paper's workloads (Table 1): clustered float32 and uint8 vectors.
"""
import threading

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
import synth
from parity_checks import (RTOL, _adc_ref, _check_topk, _expanded_magnitude, _l2_ref,
                           _lowp_adc_bound, _lowp_lut_bound)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_16576_b300 as m
    return m


def _oracle_lists(parts):
    return oracle.lists_from_parts(parts["primary"], parts["rep_off"], parts["rep_ids"],
                                   parts["nlist"])


# ---------------------------------------------------------------------------
# fixtures
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def f32_small(fa):
    """100k float32 d=128 vectors, 256 lists, M=16, nprobe 8, k 10 (the plain
    FP32 workload), 100 queries."""
    w = synth.plain_f32_100k()
    base = w.mix.base(w.n)
    q = w.mix.queries(w.nq)
    ix = fa.fa_build_index(base, fa.build_params(nlist=w.nlist, M=w.M, kmeans_iters=8,
                                                 raw_location=fa.FA_RAW_DEVICE))
    parts = ix.parts()
    off, ids = _oracle_lists(parts)
    return dict(w=w, base=base, q=q, ix=ix, parts=parts, off=off, ids=ids)


@pytest.fixture(scope="module")
def u8_repl(fa):
    """uint8 d=128 vectors with Eq. 2 replication (up to 4 lists per vector),
    raw vectors in pinned host memory."""
    mix = synth.Mixture(128, 16, 8.0, kind="u8")
    base = mix.base(30_000)
    q = mix.queries(40)
    ix = fa.fa_build_index(base, fa.build_params(nlist=64, M=32, kmeans_iters=6, repl_eps=0.08,
                                                 max_lists_per_vec=4,
                                                 raw_location=fa.FA_RAW_HOST_PINNED))
    parts = ix.parts()
    assert parts["rep_off"][-1] > 0, "the build produced no replicas"
    off, ids = _oracle_lists(parts)
    return dict(base=base, q=q, ix=ix, parts=parts, off=off, ids=ids)


# ---------------------------------------------------------------------------
# step 2: coarse probe
# ---------------------------------------------------------------------------

def test_coarse_probe_matches_oracle(fa, f32_small):
    s = f32_small
    npb = 8
    got = fa.fa_debug_probes(s["ix"], s["q"], npb)
    ref, d2 = oracle.coarse(s["q"], s["parts"]["centroids"], npb + 1, with_d2=True)
    for i in range(s["q"].shape[0]):
        if got[i].tolist() != ref[i, :npb].tolist():
            # only a near tie at the boundary may reorder the probe set
            assert abs(d2[i, npb] - d2[i, npb - 1]) <= 1e-5 * d2[i, npb - 1], i
            assert set(got[i].tolist()) - set(ref[i, :npb + 1].tolist()) == set(), i


# ---------------------------------------------------------------------------
# step 1: LUT
# ---------------------------------------------------------------------------

def test_lut_f32_matches_oracle(fa, f32_small):
    s = f32_small
    for i in range(5):
        got = fa.fa_debug_lut(s["ix"], s["q"][i])
        ref = oracle.lut(s["q"][i], s["parts"]["codebooks"])
        np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-2)


@pytest.mark.parametrize("which", ["f32", "u8"])
def test_lut_tc_matches_oracle(fa, f32_small, u8_repl, which):
    """BF16 tensor-core LUT (hi/lo split, FP32 accumulation) against the FP64
    table: within 4e-5 of the magnitude of the expanded form's terms."""
    s = f32_small if which == "f32" else u8_repl
    p = fa.search_params(lut_gemm=fa.FA_GEMM_BF16_TC)
    for i in range(4):
        got = fa.fa_debug_lut(s["ix"], s["q"][i], p).astype(np.float64)
        ref = oracle.lut(s["q"][i], s["parts"]["codebooks"])
        tol = 4e-5 * _expanded_magnitude(s["q"][i], s["parts"]["codebooks"]) + 1e-3
        assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) - tol)


@pytest.mark.parametrize("gemm", ["SIMT_F32", "BF16_TC"])
@pytest.mark.parametrize("prec,rel", [("F16", 2.0 ** -11), ("FP8", 2.0 ** -4)])
def test_lut_lowp_error_bound(fa, u8_repl, prec, rel, gemm):
    """FP16 / FP8 table: each entry is within half a unit in the last place of
    its stored residual (times its subspace's scale) of the FP64 value, plus
    the tensor-core form's rounding when the table comes from the GEMM."""
    s = u8_repl
    p = fa.search_params(lut_prec=getattr(fa, "FA_LUT_" + prec), lut_gemm=getattr(fa, "FA_GEMM_" + gemm))
    for i in range(4):
        got = fa.fa_debug_lut(s["ix"], s["q"][i], p).astype(np.float64)
        ref = oracle.lut(s["q"][i], s["parts"]["codebooks"])
        resid = ref - ref.min(axis=1, keepdims=True)
        # half-ulp of the stored value (relative), an FP32 rounding margin, and
        # the FP8 subnormal step (2^-9 of the scale) for tiny residuals
        scale = resid.max(axis=1, keepdims=True) / (65504.0 if prec == "F16" else 448.0)
        bound = resid * rel + 1e-5 * np.abs(ref) + scale * (2.0 ** -9 if prec == "FP8" else 2.0 ** -24) + 1e-3
        if gemm == "BF16_TC":
            bound = bound + 4e-5 * _expanded_magnitude(s["q"][i], s["parts"]["codebooks"]) * (1 + rel)
        assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) - bound)


@pytest.mark.parametrize("prec,gemm", [("F32", "SIMT_F32"), ("F16", "SIMT_F32"), ("FP8", "SIMT_F32"),
                                       ("F32", "BF16_TC"), ("F16", "BF16_TC"), ("FP8", "BF16_TC")])
def test_adc_equals_sum_of_lut_entries(fa, u8_repl, prec, gemm):
    """Invariant of Eq. 1: every returned ADC distance is the sum of the M
    entries of the query's table (as the scan reads it) picked by the
    vector's codes, up to FP32 summation order."""
    s = u8_repl
    p = fa.search_params(lut_prec=getattr(fa, "FA_LUT_" + prec), lut_gemm=getattr(fa, "FA_GEMM_" + gemm))
    q = s["q"][:8]
    probes = oracle.coarse(q, s["parts"]["centroids"], 8)
    gi, gd = fa.fa_search_ex(s["ix"], q, 50, 8, p, probes=probes)
    codes = s["parts"]["codes"]
    M = codes.shape[1]
    for i in range(q.shape[0]):
        lut = fa.fa_debug_lut(s["ix"], q[i], p).astype(np.float64)
        ok = gi[i] >= 0
        ref = lut[np.arange(M)[None, :], codes[gi[i][ok]]].sum(1)
        np.testing.assert_allclose(gd[i][ok], ref, rtol=2e-6, atol=1e-3)


@pytest.mark.parametrize("which", ["f32", "u8"])
def test_coarse_probe_tc_matches_oracle(fa, f32_small, u8_repl, which):
    """Tensor-core coarse probe: the oracle's probe list except where the
    boundary distances are closer than the expanded form's rounding."""
    s = f32_small if which == "f32" else u8_repl
    npb = 8
    got = fa.fa_debug_probes(s["ix"], s["q"], npb, fa.search_params(probe_gemm=fa.FA_GEMM_BF16_TC))
    ref, d2 = oracle.coarse(s["q"], s["parts"]["centroids"], npb + 4, with_d2=True)
    cent = s["parts"]["centroids"].astype(np.float64)
    for i in range(s["q"].shape[0]):
        if got[i].tolist() == ref[i, :npb].tolist():
            continue
        mag = (s["q"][i].astype(np.float64) ** 2).sum() + (cent ** 2).sum(1).max()
        gd2 = ((cent[got[i]] - s["q"][i].astype(np.float64)) ** 2).sum(1)
        # every chosen list is within the rounding of the boundary distance
        assert np.all(gd2 <= d2[i, npb - 1] + 4e-5 * mag), i


def _probe_index(fa, d, nlist, nq, seed):
    """An index over clustered centroids (d <= 128) that only the probe reads."""
    mix = synth.Mixture(d, 32, 4.0, lo=-20.0, hi=20.0, seed=seed)
    cent = mix.base(nlist)
    M = {128: 32, 96: 48, 64: 16, 32: 8}[d]
    cb = np.zeros((M, 256, d // M), np.float32)
    codes = np.zeros((64, M), np.uint8)
    prim = (np.arange(64) % nlist).astype(np.int32)
    return fa.fa_index_from_parts(cent, cb, codes, prim), cent, mix.queries(nq)


@pytest.mark.parametrize("d,nlist,nq,n", [
    (128, 1000, 300, 1), (128, 1000, 300, 8), (128, 1000, 300, 33), (128, 1000, 300, 64),
    (128, 1000, 300, 100), (128, 1000, 300, 256), (128, 1000, 300, 512),
    (96, 5000, 1000, 40), (64, 8192, 2000, 128), (32, 300, 129, 200), (128, 16384, 1, 64)])
def test_fused_tc_probe_shapes(fa, d, nlist, nq, n):
    """Fused tensor-core probe (distances and top-nprobe in one kernel) over
    ragged query and centroid tiles, CTA ranges that cross query tiles, and
    queues that fill and compact: n distinct lists per query, in distance
    order, each within the expanded form's rounding of the oracle's n-th
    distance, and every oracle list it leaves out at that boundary."""
    ix, cent, q = _probe_index(fa, d, nlist, nq, seed=d + nlist + n)
    got = fa.fa_debug_probes(ix, q, n, fa.search_params(probe_gemm=fa.FA_GEMM_BF16_TC))
    ref, d2 = oracle.coarse(q, cent, n, with_d2=True)
    c64 = cent.astype(np.float64)
    cn = (c64 ** 2).sum(1)
    for i in range(nq):
        g = got[i]
        assert g.min() >= 0 and g.max() < nlist and len(set(g.tolist())) == n, i
        q64 = q[i].astype(np.float64)
        tol = 4e-5 * ((q64 ** 2).sum() + cn.max())
        gd = ((c64[g] - q64) ** 2).sum(1)
        kth = d2[i, n - 1]
        assert np.all(gd <= kth + tol), i
        assert np.all(np.diff(gd) >= -tol), i
        missing = np.array(sorted(set(ref[i].tolist()) - set(g.tolist())), dtype=np.int64)
        if missing.size:
            assert np.all(((c64[missing] - q64) ** 2).sum(1) >= kth - tol), i


# ---------------------------------------------------------------------------
# steps 3-5: gather + dedup (bit-exact)
# ---------------------------------------------------------------------------

def test_candidates_bit_exact_with_replication(fa, u8_repl):
    s = u8_repl
    nl = s["parts"]["nlist"]
    rng = np.random.default_rng(5)
    for t in range(30):
        npb = int(rng.integers(1, 24))
        probes = rng.choice(nl, size=npb, replace=False).astype(np.int32)
        got = fa.fa_debug_candidates(s["ix"], probes=probes)
        ref, gathered = oracle.candidates(probes, s["off"], s["ids"])
        assert got.dtype == np.int64
        assert got.tolist() == ref.astype(np.int64).tolist(), t
    # every list probed: each vector exactly once
    got = fa.fa_debug_candidates(s["ix"], probes=np.arange(nl, dtype=np.int32))
    assert got.tolist() == list(range(s["parts"]["n"]))


def test_candidate_counts_in_stats(fa, u8_repl):
    s = u8_repl
    nl = s["parts"]["nlist"]
    probes = np.tile(np.arange(12, dtype=np.int32), (3, 1))
    _, _, st = fa.fa_search_ex(s["ix"], s["q"][:3], 10, 12, probes=probes, stats=True)
    ref, gathered = oracle.candidates(probes[0], s["off"], s["ids"])
    assert np.all(st[:, 0] == gathered) and np.all(st[:, 1] == ref.shape[0])
    _, _, st = fa.fa_search_ex(s["ix"], s["q"][:1], 10, nl, probes=np.arange(nl)[None], stats=True)
    assert st[0, 1] == s["parts"]["n"] and st[0, 0] == s["off"][-1]


# ---------------------------------------------------------------------------
# steps 6-7: ADC + top-k through fa_search_ex
# ---------------------------------------------------------------------------

def _search_vs_oracle(fa, s, k, npb, params=None, nq=None, rerank=0):
    q = s["q"][:nq] if nq else s["q"]
    probes = oracle.coarse(q, s["parts"]["centroids"], npb)
    gi, gd = fa.fa_search_ex(s["ix"], q, k, npb, params, probes=probes)
    kk = rerank if rerank else k + 1
    oi, od = oracle.search(q, s["parts"]["centroids"], s["parts"]["codebooks"], s["parts"]["codes"],
                           s["off"], s["ids"], npb, kk, probes=probes)
    return gi, gd, oi, od


@pytest.mark.parametrize("k", [1, 10, 100, 300, 1000])
def test_search_given_probes_matches_oracle(fa, f32_small, k):
    """k <= 256 runs the per-warp top-n, larger k the CTA-wide top-n."""
    s = f32_small
    gi, gd, oi, od = _search_vs_oracle(fa, s, k, 8)
    for i in range(gi.shape[0]):
        _check_topk(gi[i], gd[i], oi[i, :k], od[i, :k], od[i, k], k, what=str(i),
                    ref_of=_adc_ref(s["q"][i], s["parts"]))
        # rows ascending by (distance, id)
        fin = np.isfinite(gd[i])
        keys = list(zip(gd[i][fin].tolist(), gi[i][fin].tolist()))
        assert keys == sorted(keys)


@pytest.mark.parametrize("k", [10, 600])
def test_search_with_replication_matches_oracle(fa, u8_repl, k):
    s = u8_repl
    gi, gd, oi, od = _search_vs_oracle(fa, s, k, 16)
    for i in range(gi.shape[0]):
        _check_topk(gi[i], gd[i], oi[i, :k], od[i, :k], od[i, k], k, what=str(i),
                    ref_of=_adc_ref(s["q"][i], s["parts"]))
        assert len(set(gi[i].tolist())) == k  # no duplicate ids


@pytest.mark.parametrize("k", [4097, 6000, 16384])
def test_large_topn_matches_oracle(fa, f32_small, k):
    """Top-n above 4096 (the re-rank depths that recall@10 = 0.9 needs): the
    CTA-wide selection keeps its top-n beside the LUT with a staging region
    smaller than the top-n once both do not fit in shared memory (nprobe 64 of
    256 lists: about 25k distinct candidates, so the threshold filter and many
    merges run)."""
    s = f32_small
    gi, gd, oi, od = _search_vs_oracle(fa, s, k, 64, nq=6)
    for i in range(gi.shape[0]):
        _check_topk(gi[i], gd[i], oi[i, :k], od[i, :k], od[i, k], k, what=str(i),
                    ref_of=_adc_ref(s["q"][i], s["parts"]))
        fin = np.isfinite(gd[i])
        keys = list(zip(gd[i][fin].tolist(), gi[i][fin].tolist()))
        assert keys == sorted(keys)
        assert len(set(gi[i][fin].tolist())) == int(fin.sum())


def test_end_to_end_recall_matches_oracle(fa, f32_small):
    """Whole path (coarse probe included) on the plain FP32 workload: recall@10
    against brute force within 0.005 of the oracle's."""
    s = f32_small
    w = s["w"]
    gi, gd = fa.fa_search(s["ix"], s["q"], w.k, w.nprobe)
    oi, od = oracle.search(s["q"], s["parts"]["centroids"], s["parts"]["codebooks"],
                           s["parts"]["codes"], s["off"], s["ids"], w.nprobe, w.k)
    ti, td = oracle.knn(s["q"], s["base"], w.k)
    r_gpu = oracle.recall_at(gi, ti, td, at=w.k)
    r_ora = oracle.recall_at(oi, ti, td, at=w.k)
    assert abs(r_gpu - r_ora) <= 0.005, (r_gpu, r_ora)


def test_persistent_and_device_buffers_match(fa, f32_small):
    import torch
    s = f32_small
    gi, gd = fa.fa_search(s["ix"], s["q"], 10, 8)
    pi, pd = fa.fa_search_ex(s["ix"], s["q"], 10, 8, fa.search_params(flags=fa.FA_PERSISTENT))
    assert np.array_equal(gi, pi) and np.array_equal(gd, pd)
    qd = torch.as_tensor(s["q"], device="cuda")
    di, dd = fa.fa_search_ex(s["ix"], qd, 10, 8)
    torch.cuda.synchronize()
    assert np.array_equal(gi, di.cpu().numpy()) and np.array_equal(gd, dd.cpu().numpy())


@pytest.mark.parametrize("k,rerank", [(10, 0), (100, 0), (10, 600)])
def test_autotune_variants_agree_and_keep_results(fa, u8_repl, k, rerank):
    """The autotuner times every scan launch shape (it fails if any returns
    different rows) and the tuned index returns the same results."""
    s = u8_repl
    p = fa.search_params(rerank_n=rerank, rerank_eps=-1.0, lut_prec=fa.FA_LUT_F16,
                         lut_gemm=fa.FA_GEMM_BF16_TC)
    before = fa.fa_search_ex(s["ix"], s["q"], k, 16, p)
    r = fa.fa_autotune(s["ix"], s["q"], k, 16, p)
    assert len(r["variants"]) == (8 if k + rerank <= 256 else 2)
    assert all(v["scan_ms"] > 0 for v in r["variants"])
    after = fa.fa_search_ex(s["ix"], s["q"], k, 16, p)
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])


@pytest.fixture(scope="module")
def zipf_small(fa):
    """Uneven lists: 64 lists with Zipf(1.1) sizes over 60k vectors (the
    largest list holds about a third of them), random codes and codebooks."""
    rng = np.random.default_rng(33)
    n, d, M, nlist = 60_000, 32, 16, 64
    sizes = synth.zipf_sizes(nlist, n)
    primary = np.repeat(np.arange(nlist, dtype=np.int32), sizes)
    rng.shuffle(primary)
    cent = rng.normal(size=(nlist, d)).astype(np.float32)
    cb = rng.normal(size=(M, 256, d // M)).astype(np.float32)
    codes = rng.integers(0, 256, size=(n, M)).astype(np.uint8)
    ix = fa.fa_index_from_parts(cent, cb, codes, primary)
    parts = ix.parts()
    off, ids = _oracle_lists(parts)
    q = rng.normal(size=(200, d)).astype(np.float32)
    return dict(ix=ix, parts=parts, off=off, ids=ids, q=q, sizes=sizes)


@pytest.mark.parametrize("k", [10, 100])
def test_tiled_batching_form_on_uneven_lists(fa, zipf_small, k):
    """Persistent tiled form with per-query nprobe in 1..16 over Zipf-sized
    lists: the oracle's top-k, and the same rows as one CTA per query."""
    s = zipf_small
    rng = np.random.default_rng(k)
    nq = s["q"].shape[0]
    npq = rng.integers(1, 17, size=nq).astype(np.int32)
    probes = oracle.coarse(s["q"], s["parts"]["centroids"], 16)
    tiled = fa.fa_search_ex(s["ix"], s["q"], k, 16, fa.search_params(flags=fa.FA_PERSISTENT),
                            probes=probes, nprobe_per_query=npq)
    plain = fa.fa_search_ex(s["ix"], s["q"], k, 16, probes=probes, nprobe_per_query=npq)
    assert np.array_equal(tiled[0], plain[0]) and np.array_equal(tiled[1], plain[1])
    assert s["sizes"].max() > 0.25 * s["parts"]["n"]
    for i in range(0, nq, 7):
        oi, od = oracle.search(s["q"][i:i + 1], s["parts"]["centroids"], s["parts"]["codebooks"],
                               s["parts"]["codes"], s["off"], s["ids"], int(npq[i]), k + 1,
                               probes=probes[i:i + 1, :npq[i]])
        _check_topk(tiled[0][i], tiled[1][i], oi[0, :k], od[0, :k], od[0, k], k, what=str(i),
                    ref_of=_adc_ref(s["q"][i], s["parts"]))


@pytest.mark.parametrize("flags", ["eager_graph", "tiled_graph"])
def test_graph_capture_replays_the_search(fa, zipf_small, flags):
    """FA_GRAPH: the first call captures the kernels into a CUDA graph, later
    calls with the same buffers replay it and read the buffers' new contents."""
    import torch
    s = zipf_small
    f = fa.FA_GRAPH | (fa.FA_PERSISTENT if flags == "tiled_graph" else 0)
    p = fa.search_params(flags=f, lut_prec=fa.FA_LUT_F16, lut_gemm=fa.FA_GEMM_BF16_TC,
                         probe_gemm=fa.FA_GEMM_BF16_TC)
    ref = fa.search_params(lut_prec=fa.FA_LUT_F16, lut_gemm=fa.FA_GEMM_BF16_TC,
                           probe_gemm=fa.FA_GEMM_BF16_TC)
    qd = torch.as_tensor(s["q"], device="cuda")
    oi = torch.empty((qd.shape[0], 10), dtype=torch.int64, device="cuda")
    od = torch.empty((qd.shape[0], 10), dtype=torch.float32, device="cuda")
    for rnd in range(3):
        if rnd == 2:
            qd.mul_(-1.0)  # new query contents in the same buffer
        fa.fa_search_ex(s["ix"], qd, 10, 8, p, out_ids=oi, out_dist=od)
        torch.cuda.synchronize()
        ei, ed = fa.fa_search_ex(s["ix"], qd.cpu().numpy(), 10, 8, ref)
        assert np.array_equal(oi.cpu().numpy(), ei) and np.array_equal(od.cpu().numpy(), ed), rnd
    with pytest.raises(fa.FaError) as e:
        fa.fa_search_ex(s["ix"], s["q"], 10, 8, p)  # host buffers cannot be captured
    assert e.value.status == fa.FA_ERR_ARG


def test_build_with_given_lists(fa):
    """fa_build_index_lists keeps the caller's lists and centroids and trains
    only PQ; searches on it match the oracle on the exported parts."""
    z = synth.ZipfLists(40_000, d=32, nlist=128, ncomp=16)
    base, cent, prim = z.base(), z.centroids(), z.primary()
    ix = fa.fa_build_index_lists(base, cent, prim, fa.build_params(M=16, kmeans_iters=4))
    parts = ix.parts()
    assert np.array_equal(parts["primary"], prim) and np.array_equal(parts["centroids"], cent)
    q = z.queries(30)
    off, ids = _oracle_lists(parts)
    probes = oracle.coarse(q, cent, 8)
    gi, gd = fa.fa_search_ex(ix, q, 10, 8, probes=probes)
    oi, od = oracle.search(q, cent, parts["codebooks"], parts["codes"], off, ids, 8, 11, probes=probes)
    for i in range(q.shape[0]):
        _check_topk(gi[i], gd[i], oi[i, :10], od[i, :10], od[i, 10], 10, what=str(i),
                    ref_of=_adc_ref(q[i], parts))


def _serve_all(srv, n):
    got = {}
    while len(got) < n:
        rid, ids, dist, lat, st = srv.poll(timeout_us=20000)
        for j in range(rid.shape[0]):
            assert st[j] == 0
            got[int(rid[j])] = (ids[j], dist[j], lat[j])
    return got


@pytest.mark.parametrize("lowp", [False, True, "batched"])
def test_serving_result_same_alone_and_in_the_mix(fa, u8_repl, lowp):
    """Continuous batching: every request's result equals the result of the
    same query searched alone (same k, nprobe and parameters), bit for bit;
    with the batched form (FP8 table, exhaustive re-rank) every served
    distance is the oracle's exact distance of that id."""
    s = u8_repl
    tc = fa.FA_GEMM_BF16_TC
    if lowp == "batched":
        p = fa.search_params(lut_prec=fa.FA_LUT_FP8, lut_gemm=tc, probe_gemm=tc, rerank_n=50,
                             rerank_eps=-1.0, flags=fa.FA_BATCHED)
    else:
        p = fa.search_params(lut_prec=fa.FA_LUT_F16, lut_gemm=tc, probe_gemm=tc, rerank_n=50,
                             rerank_eps=0.0) if lowp else fa.search_params()
    rng = np.random.default_rng(4)
    n = 120
    q = np.concatenate([s["q"]] * 3)[:n]
    ks = rng.choice([1, 10, 32], size=n).astype(np.int32)
    nps = rng.integers(1, 33, size=n).astype(np.int32)
    srv = fa.Server(s["ix"], p, max_batch=16, window_us=300, slots=3, kmax=32, nprobe_max=32)
    try:
        rid = np.concatenate([srv.submit(q[i:i + 10], ks[i:i + 10], nps[i:i + 10])
                              for i in range(0, n, 10)])
        got = _serve_all(srv, n)
        st = srv.stats()
        assert st.requests == n and st.batches >= n // 16
    finally:
        srv.close()
    for i in range(n):
        ids, dist, _ = got[int(rid[i])]
        ai, ad = fa.fa_search_ex(s["ix"], q[i:i + 1], int(ks[i]), int(nps[i]), p)
        assert np.array_equal(ids[:ks[i]], ai[0]) and np.array_equal(dist[:ks[i]], ad[0]), i
        assert np.all(ids[ks[i]:] == -1)
    if lowp == "batched":
        for i in range(n):
            ids, dist, _ = got[int(rid[i])]
            k = int(ks[i])
            ref = oracle.exact(q[i], s["parts"]["raw"], ids[:k].astype(np.int64))
            assert np.array_equal(dist[:k], ref.astype(np.float32)) and np.all(np.diff(dist[:k]) >= 0), i
        return
    # each request against the oracle: the served row equals the row searched
    # alone (above), and that row is checked here against the FP64 oracle
    compared = 0
    for i in range(n):
        ids, dist, _ = got[int(rid[i])]
        k, npb = int(ks[i]), int(nps[i])
        gprobe = fa.fa_debug_probes(s["ix"], q[i:i + 1], npb, p)[0]
        oprobe = oracle.coarse(q[i:i + 1], s["parts"]["centroids"], npb)[0]
        if sorted(gprobe.tolist()) != sorted(oprobe.tolist()):
            continue  # a near tie in the probe set changes the scanned lists
        if not lowp:
            oi, od = oracle.search(q[i:i + 1], s["parts"]["centroids"], s["parts"]["codebooks"],
                                   s["parts"]["codes"], s["off"], s["ids"], npb, k + 1,
                                   probes=oprobe[None])
            _check_topk(ids[:k], dist[:k], oi[0, :k], od[0, :k], od[0, k], k, what=str(i),
                        ref_of=_adc_ref(q[i], s["parts"]))
        else:
            # the FP16 table's ADC top-50 (each distance within the table's
            # error bound of the oracle's), handed to the oracle's Algorithm 1,
            # must give the served ids and exact distances
            pa = fa.search_params(lut_prec=fa.FA_LUT_F16, lut_gemm=fa.FA_GEMM_BF16_TC,
                                  probe_gemm=fa.FA_GEMM_BF16_TC)
            an_i, an_d = fa.fa_search_ex(s["ix"], q[i:i + 1], 50, npb, pa, probes=gprobe[None])
            tasks = an_i[0][an_i[0] >= 0]
            bound = _lowp_adc_bound(q[i], s["parts"], "F16", True)(tasks)
            ref = _adc_ref(q[i], s["parts"])(tasks)
            assert np.all(np.abs(an_d[0][:len(tasks)] - ref) <= bound), i
            if len(np.unique(an_d[0][:len(tasks)])) != len(tasks):
                continue  # equal ADC keys: the re-rank's order among them is the GPU's
            oi, od, _ = oracle.rerank(q[i], s["parts"]["raw"], tasks, k, batch=32, eps=0.0, beta=2)
            assert ids[:k].tolist() == oi.tolist(), i
            assert dist[:k].tolist() == od.astype(np.float32).tolist(), i
        compared += 1
    assert compared >= n // 2, compared


def test_serving_admits_by_slots(fa, f32_small):
    """One memory slot: batches run one after another, every request completes."""
    s = f32_small
    srv = fa.Server(s["ix"], None, max_batch=8, window_us=50, slots=1, kmax=10, nprobe_max=8)
    try:
        q = np.concatenate([s["q"]] * 6)
        rid = srv.submit(q, 10, 8)
        got = _serve_all(srv, q.shape[0])
        st = srv.stats()
        assert st.slots == 1 and st.batches >= q.shape[0] // 8
        assert all(got[int(r)][2] > 0 for r in rid)
    finally:
        srv.close()
    ref = fa.fa_search(s["ix"], q[:5], 10, 8)
    for i in range(5):
        assert np.array_equal(got[int(rid[i])][0], ref[0][i])


def test_per_query_k_and_nprobe(fa, f32_small):
    s = f32_small
    q = s["q"][:20]
    rng = np.random.default_rng(9)
    kq = rng.integers(1, 11, size=20).astype(np.int32)
    npq = rng.integers(1, 9, size=20).astype(np.int32)
    gi, gd = fa.fa_search_ex(s["ix"], q, 10, 8, k_per_query=kq, nprobe_per_query=npq)
    probes = oracle.coarse(q, s["parts"]["centroids"], 8)
    for i in range(20):
        oi, od = oracle.search(q[i:i + 1], s["parts"]["centroids"], s["parts"]["codebooks"],
                               s["parts"]["codes"], s["off"], s["ids"], int(npq[i]), int(kq[i]) + 1,
                               probes=probes[i:i + 1, :npq[i]])
        gprobe = fa.fa_debug_probes(s["ix"], q[i:i + 1], 8)[0]
        if gprobe[:npq[i]].tolist() != probes[i, :npq[i]].tolist():
            continue  # a near tie in the probe order changes the scanned lists
        _check_topk(gi[i, :kq[i]], gd[i, :kq[i]], oi[0, :kq[i]], od[0, :kq[i]], od[0, kq[i]], kq[i],
                    ref_of=_adc_ref(q[i], s["parts"]))
        assert np.all(gi[i, kq[i]:] == -1) and np.all(np.isinf(gd[i, kq[i]:]))


# ---------------------------------------------------------------------------
# invariants and edge cases on hand-made indexes
# ---------------------------------------------------------------------------

def _identity_parts(rng, n, d, M, nlist, rep_frac):
    x = (rng.normal(size=(n, d)) * 6).astype(np.float32)
    dsub = d // M
    cb = np.zeros((M, 256, dsub), np.float32)
    for m in range(M):
        cb[m, :n] = x[:, m * dsub:(m + 1) * dsub]
    codes = np.repeat(np.arange(n, dtype=np.uint8)[:, None], M, axis=1)
    # the last quarter of the lists gets no primary members
    primary = rng.integers(0, nlist - nlist // 4, size=n).astype(np.int32)
    rep = [[] for _ in range(nlist)]
    for v in np.nonzero(rng.random(n) < rep_frac)[0]:
        for l in rng.choice(nlist, size=3, replace=False):
            if l != primary[v]:
                rep[l].append(int(v))
    rep_off = np.zeros(nlist + 1, np.int64)
    rep_off[1:] = np.cumsum([len(a) for a in rep])
    rep_ids = np.array([v for a in rep for v in a], np.int64)
    cent = rng.normal(size=(nlist, d)).astype(np.float32)
    return x, cent, cb, codes, primary, rep_off, rep_ids


@pytest.mark.parametrize("M", [8, 16, 32, 48, 64])
def test_identity_codebook_full_probe_equals_knn(fa, M):
    """Every vector is its own PQ centroid and every list is probed: the GPU's
    IVF-PQ top-k is exact k-NN (pins gather, dedup, LUT, ADC, top-k)."""
    rng = np.random.default_rng(100 + M)
    d = 2 * M if M != 64 else 128
    x, cent, cb, codes, primary, ro, ri = _identity_parts(rng, 250, d, M, 16, 0.3)
    ix = fa.fa_index_from_parts(cent, cb, codes, primary, ro, ri)
    q = (rng.normal(size=(12, d)) * 6).astype(np.float32)
    gi, gd = fa.fa_search(ix, q, 10, 16)
    ti, td = oracle.knn(q, x, 11)
    for i in range(q.shape[0]):
        # the identity codebook makes the ADC distance the exact distance
        _check_topk(gi[i], gd[i], ti[i, :10], td[i, :10], td[i, 10], 10, what="M%d q%d" % (M, i),
                    ref_of=_l2_ref(q[i], x))


def test_fewer_candidates_than_k_and_empty_lists(fa):
    rng = np.random.default_rng(3)
    x, cent, cb, codes, primary, ro, ri = _identity_parts(rng, 40, 32, 16, 8, 0.0)
    ix = fa.fa_index_from_parts(cent, cb, codes, primary, ro, ri)
    counts = np.bincount(primary, minlength=8)
    empty = int(np.argmin(counts))
    assert counts[empty] == 0
    small = int(np.argmin(np.where(counts > 0, counts, 10 ** 9)))
    q = x[:3]
    probes = np.array([[empty, small]] * 3, np.int32)
    k = int(counts[small]) + 5
    gi, gd = fa.fa_search_ex(ix, q, k, 2, probes=probes)
    members = sorted(np.nonzero(primary == small)[0].tolist())
    for i in range(3):
        assert sorted(gi[i, :counts[small]].tolist()) == members
        assert np.all(gi[i, counts[small]:] == -1) and np.all(np.isinf(gd[i, counts[small]:]))
    # only empty lists probed: every row is padding
    gi, gd = fa.fa_search_ex(ix, q, 4, 1, probes=np.full((3, 1), empty, np.int32))
    assert np.all(gi == -1) and np.all(np.isinf(gd))


def test_argument_errors_and_empty_batch(fa, f32_small):
    s = f32_small
    gi, gd = fa.fa_search(s["ix"], s["q"][:0], 10, 8)
    assert gi.shape == (0, 10)
    with pytest.raises(fa.FaError) as e:
        fa.fa_search(s["ix"], s["q"][:, :64], 10, 8)
    assert e.value.status == fa.FA_ERR_ARG
    with pytest.raises(fa.FaError) as e:
        fa.fa_search(s["ix"], s["q"], 0, 8)
    assert e.value.status == fa.FA_ERR_ARG
    # nprobe above nlist is clamped, not an error
    gi, gd = fa.fa_search(s["ix"], s["q"][:2], 5, 100000)
    assert gi.shape == (2, 5)
    bad = np.full((2, 8), 99999, np.int32)
    with pytest.raises(fa.FaError) as e:
        fa.fa_search_ex(s["ix"], s["q"][:2], 5, 8, probes=bad)
    assert e.value.status == fa.FA_ERR_ARG
    # the index stays usable after argument errors
    gi2, _ = fa.fa_search(s["ix"], s["q"][:2], 5, 8)
    assert gi2.shape == (2, 5)


# ---------------------------------------------------------------------------
# step 8: Algorithm 1 on the GPU
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("eps,beta,batch,n", [(0.0, 2, 32, 100), (-1.0, 1, 32, 100),
                                              (1.0, 1, 32, 100), (0.1, 1, 16, 100),
                                              (0.0, 3, 8, 100), (-1.0, 1, 32, 1000),
                                              (0.0, 2, 256, 1000)])
def test_rerank_matches_oracle(fa, u8_repl, eps, beta, batch, n):
    s = u8_repl
    k, npb = 10, 16
    q = s["q"][:24]
    probes = oracle.coarse(q, s["parts"]["centroids"], npb)
    p = fa.search_params(rerank_n=n, rerank_batch=batch, rerank_beta=beta, rerank_eps=eps)
    gi, gd, st = fa.fa_search_ex(s["ix"], q, k, npb, p, probes=probes, stats=True)
    oi, od, ost = oracle.search(q, s["parts"]["centroids"], s["parts"]["codebooks"],
                                s["parts"]["codes"], s["off"], s["ids"], npb, k, raw=s["parts"]["raw"],
                                probes=probes, rerank_n=n, batch=batch, eps=eps, beta=beta, stats=True)
    # re-rank inputs (the ADC top-n) may differ at an ADC near tie; compare
    # where the GPU's ADC top-n equals the oracle's
    an_i, an_d = fa.fa_search_ex(s["ix"], q, n, npb, probes=probes)
    ao_i, ao_d = oracle.search(q, s["parts"]["centroids"], s["parts"]["codebooks"],
                               s["parts"]["codes"], s["off"], s["ids"], npb, n, probes=probes)
    compared = 0
    for i in range(q.shape[0]):
        if an_i[i].tolist() != ao_i[i].tolist():
            continue
        compared += 1
        # uint8 data and integral queries: exact distances are integers in FP32
        assert gd[i].tolist() == od[i].astype(np.float32).tolist(), i
        assert gi[i].tolist() == oi[i].tolist(), i
        assert st[i, 2] == ost[i, 2], (i, st[i], ost[i])
    assert compared >= q.shape[0] // 2


@pytest.mark.parametrize("shift", [0.0, 0.3, -1.0])
def test_rerank_uint8_rows_any_query(fa, u8_repl, shift):
    """uint8 raw rows: integral queries in 0..255 take the integer (dp4a)
    distance form, other queries (fractional, or below 0) the float form;
    both give the oracle's exact distances (the integer form exactly)."""
    s = u8_repl
    k, npb, n = 10, 16, 200
    q = (s["q"][:16] + np.float32(shift)).astype(np.float32)
    probes = oracle.coarse(q, s["parts"]["centroids"], npb)
    p = fa.search_params(rerank_n=n, rerank_eps=-1.0)
    gi, gd = fa.fa_search_ex(s["ix"], q, k, npb, p, probes=probes)
    an_i, _ = fa.fa_search_ex(s["ix"], q, n, npb, probes=probes)
    for i in range(q.shape[0]):
        tasks = an_i[i][an_i[i] >= 0]
        oi, od, _ = oracle.rerank(q[i], s["parts"]["raw"], tasks, k, batch=32, eps=-1.0, beta=1)
        if shift == 0.0:
            assert gd[i].tolist() == od.astype(np.float32).tolist(), i
            assert gi[i].tolist() == oi.tolist(), i
        else:
            _check_topk(gi[i], gd[i], oi, od, od[-1], k, what=str(i),
                        ref_of=_l2_ref(q[i], s["parts"]["raw"]))


@pytest.fixture(scope="module")
def u8_dev(fa):
    """uint8 d=128 vectors with raw rows in HBM (internal order), where an
    exhaustive re-rank of a top-n above 256 runs fused into the scan."""
    mix = synth.Mixture(128, 16, 8.0, kind="u8")
    base = mix.base(40_000)
    q = mix.queries(24)
    ix = fa.fa_build_index(base, fa.build_params(nlist=64, M=32, kmeans_iters=6,
                                                 raw_location=fa.FA_RAW_DEVICE))
    parts = ix.parts()
    off, ids = _oracle_lists(parts)
    return dict(base=base, q=q, ix=ix, parts=parts, off=off, ids=ids)


@pytest.mark.parametrize("shift,sigma", [(0.0, 4.0), (0.3, 4.0), (0.0, -1000.0)])
@pytest.mark.parametrize("n", [1000, 3000])
def test_fused_exhaustive_rerank_matches_oracle(fa, u8_dev, n, shift, sigma):
    """Exhaustive Algorithm 1 (eps < 0) over a top-n above 256 with raw rows
    in HBM runs inside the selecting scan: integral queries take the integer
    distance form, shifted ones the float form; with the threshold estimate
    forced low (sigma -1000) every query is handed back and re-ranked by the
    separate kernel over the device-side list. The GPU's own ADC top-n
    (checked against the oracle's as a set) fed to the oracle's Algorithm 1
    must give the GPU's ids, distances and mini-batch counts."""
    s = u8_dev
    k, npb = 10, 24
    q = (s["q"] + np.float32(shift)).astype(np.float32)
    probes = oracle.coarse(q, s["parts"]["centroids"], npb)
    p = fa.search_params(rerank_n=n, rerank_batch=32, rerank_eps=-1.0, lut_prec=fa.FA_LUT_F16,
                         lut_gemm=fa.FA_GEMM_BF16_TC)
    fa.fa_debug_tau_sigma(sigma)
    try:
        gi, gd, st = fa.fa_search_ex(s["ix"], q, k, npb, p, probes=probes, stats=True)
        pa = fa.search_params(lut_prec=fa.FA_LUT_F16, lut_gemm=fa.FA_GEMM_BF16_TC)
        an_i, an_d = fa.fa_search_ex(s["ix"], q, n, npb, pa, probes=probes)
    finally:
        fa.fa_debug_tau_sigma(4.0)
    for i in range(q.shape[0]):
        tasks = an_i[i][an_i[i] >= 0]
        oi, od, nb = oracle.rerank(q[i], s["parts"]["raw"], tasks, k, batch=32, eps=-1.0, beta=1)
        if shift == 0.0:
            assert gd[i].tolist() == od.astype(np.float32).tolist(), i
            assert gi[i].tolist() == oi.tolist(), i
        else:
            _check_topk(gi[i], gd[i], oi, od, od[-1], k, what=str(i),
                        ref_of=_l2_ref(q[i], s["parts"]["raw"]))
        assert st[i, 2] == nb and st[i, 3] == len(tasks), (i, st[i], nb)


@pytest.mark.parametrize("k,sigma", [(600, -1000.0), (600, 44.0), (600, 150.0),
                                     (4097, -1000.0), (4097, 125.0), (4097, 150.0)])
def test_large_topn_exact_whatever_the_estimate(fa, f32_small, k, sigma):
    """The sampled threshold estimate is only a filter. Forced far below the
    true n-th distance (sigma -1000), fewer than n keys pass it and every
    query is scanned again without it. Set a little high (sigma 44 for n 600,
    125 for n 4097, on about 25k candidates), more keys pass than the two
    shared-memory regions hold and the rest spill through the output row.
    Forced high (sigma 150), more pass than that too and the query is scanned
    again in lock-step rounds. All give the oracle's result."""
    s = f32_small
    fa.fa_debug_tau_sigma(sigma)
    try:
        gi, gd, oi, od = _search_vs_oracle(fa, s, k, 64, nq=6)
    finally:
        fa.fa_debug_tau_sigma(4.0)
    for i in range(gi.shape[0]):
        _check_topk(gi[i], gd[i], oi[i, :k], od[i, :k], od[i, k], k, what=str(i),
                    ref_of=_adc_ref(s["q"][i], s["parts"]))


@pytest.mark.parametrize("eps,beta,n", [(-1.0, 1, 8192), (-1.0, 1, 16384), (0.0, 2, 16384)])
def test_deep_rerank_matches_oracle(fa, f32_small, eps, beta, n):
    """Algorithm 1 over 8192 or 16384 ADC candidates (raw vectors in HBM).
    FP32 and FP64 ADC order near ties differently somewhere in lists this
    long, so the GPU's own ADC top-n (checked against the oracle's as a set)
    is handed to the oracle's Algorithm 1, which must reproduce the GPU's
    re-ranked ids, distances and mini-batch count."""
    s = f32_small
    k, npb = 10, 64
    q = s["q"][:6]
    probes = oracle.coarse(q, s["parts"]["centroids"], npb)
    p = fa.search_params(rerank_n=n, rerank_batch=32, rerank_beta=beta, rerank_eps=eps)
    gi, gd, st = fa.fa_search_ex(s["ix"], q, k, npb, p, probes=probes, stats=True)
    an_i, an_d = fa.fa_search_ex(s["ix"], q, n, npb, probes=probes)
    ao_i, ao_d = oracle.search(q, s["parts"]["centroids"], s["parts"]["codebooks"],
                               s["parts"]["codes"], s["off"], s["ids"], npb, n + 1, probes=probes)
    for i in range(q.shape[0]):
        _check_topk(an_i[i], an_d[i], ao_i[i, :n], ao_d[i, :n], ao_d[i, n], n, what=str(i),
                    ref_of=_adc_ref(q[i], s["parts"]))
        tasks = an_i[i][an_i[i] >= 0]
        oi, od, nb = oracle.rerank(q[i], s["parts"]["raw"], tasks, k, batch=32, eps=eps, beta=beta)
        assert gi[i].tolist() == oi.tolist(), i
        np.testing.assert_allclose(gd[i], od, rtol=RTOL, atol=1e-3)
        assert st[i, 2] == nb, (i, st[i], nb)


@pytest.mark.parametrize("lowp", [False, True])
def test_pipelined_rerank_equals_serial(fa, u8_repl, lowp):
    """A batch of >= 4096 queries re-ranked from pinned host memory is scanned
    and re-ranked in overlapping chunks on two streams; every id, distance and
    per-query statistic equals the serial order's (FA_SERIAL), on a ragged
    batch with per-query k and nprobe."""
    s = u8_repl
    q = synth.Mixture(128, 16, 8.0, kind="u8").queries(5003).astype(np.float32)
    kq = synth.uniform_ints(1, 10, q.shape[0], tag=21)
    npq = synth.uniform_ints(4, 16, q.shape[0], tag=22)
    extra = dict(lut_prec=fa.FA_LUT_F16, lut_gemm=fa.FA_GEMM_BF16_TC, probe_gemm=fa.FA_GEMM_BF16_TC) if lowp else {}
    out = []
    for flags in (0, fa.FA_SERIAL):
        p = fa.search_params(rerank_n=64, rerank_batch=16, rerank_beta=2, rerank_eps=0.0, flags=flags, **extra)
        out.append(fa.fa_search_ex(s["ix"], q, 10, 16, p, k_per_query=kq, nprobe_per_query=npq, stats=True))
    (pi, pd, pst), (si, sd, sst) = out
    assert np.array_equal(pi, si)
    assert np.array_equal(pd.view(np.uint32), sd.view(np.uint32))
    assert np.array_equal(pst, sst)
    assert np.all(pst[:, 2] >= 1)  # every query re-ranked at least one mini-batch


def test_pipelined_rerank_under_graph_capture(fa, u8_repl):
    """The pipelined search (three streams joined by events) captured into a
    CUDA graph with device buffers replays correctly, also after the query
    buffer's contents change, and equals the serial order."""
    import torch
    s = u8_repl
    q = synth.Mixture(128, 16, 8.0, kind="u8").queries(4500).astype(np.float32)
    tc = fa.FA_GEMM_BF16_TC
    base = dict(rerank_n=48, rerank_batch=16, lut_prec=fa.FA_LUT_F16, lut_gemm=tc, probe_gemm=tc)
    pg = fa.search_params(flags=fa.FA_GRAPH, **base)
    ps = fa.search_params(flags=fa.FA_SERIAL, **base)
    qd = torch.as_tensor(q, device="cuda")
    oi = torch.empty((q.shape[0], 10), dtype=torch.int64, device="cuda")
    od = torch.empty((q.shape[0], 10), dtype=torch.float32, device="cuda")
    for rnd in range(3):
        if rnd == 2:
            qd.copy_(torch.flip(qd, [0]))  # new contents, same buffer
        fa.fa_search_ex(s["ix"], qd, 10, 12, pg, out_ids=oi, out_dist=od)
        torch.cuda.synchronize()
        ei, ed = fa.fa_search_ex(s["ix"], qd.cpu().numpy(), 10, 12, ps)
        assert np.array_equal(oi.cpu().numpy(), ei), rnd
        assert np.array_equal(od.cpu().numpy().view(np.uint32), ed.view(np.uint32)), rnd


def test_rerank_device_raw_equals_pinned(fa, f32_small):
    s = f32_small
    q = s["q"][:30]
    p = fa.search_params(rerank_n=64, rerank_eps=-1.0)
    gi, gd = fa.fa_search_ex(s["ix"], q, 10, 8, p)
    # never stopping early: the result is the exact top-k of the ADC top-64
    ai, ad = fa.fa_search_ex(s["ix"], q, 64, 8)
    for i in range(q.shape[0]):
        cand = ai[i][ai[i] >= 0]
        ex = cdist(q[i:i + 1].astype(np.float64), s["base"][cand].astype(np.float64), "sqeuclidean")[0]
        order = np.lexsort((cand, ex))[:10]
        np.testing.assert_allclose(gd[i], ex[order], rtol=1e-5)
        assert set(gi[i].tolist()) == set(cand[order].tolist()) or \
            abs(ex[order][-1] - np.sort(ex)[min(10, len(ex) - 1)]) <= 1e-4 * ex[order][-1]


# ---------------------------------------------------------------------------
# lifecycle: save / load, concurrent callers
# ---------------------------------------------------------------------------

def test_save_load_roundtrip(fa, u8_repl, tmp_path):
    s = u8_repl
    path = str(tmp_path / "ix.fa")
    fa.fa_save_index(s["ix"], path)
    ix2 = fa.fa_load_index(path)
    a = fa.fa_search(s["ix"], s["q"], 10, 8)
    b = fa.fa_search(ix2, s["q"], 10, 8)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    p2 = ix2.parts()
    assert np.array_equal(p2["codes"], s["parts"]["codes"])
    assert np.array_equal(p2["raw"], s["parts"]["raw"])


def test_concurrent_callers_get_their_own_results(fa, f32_small):
    s = f32_small
    ref = [fa.fa_search(s["ix"], s["q"][i * 10:(i + 1) * 10], 10, 8) for i in range(8)]
    out = [None] * 8

    def run(i):
        out[i] = fa.fa_search(s["ix"], s["q"][i * 10:(i + 1) * 10], 10, 8)

    ts = [threading.Thread(target=run, args=(i,)) for i in range(8)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for i in range(8):
        assert np.array_equal(out[i][0], ref[i][0]) and np.array_equal(out[i][1], ref[i][1])
