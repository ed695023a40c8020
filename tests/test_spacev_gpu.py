"""The SPACEV-like workload shape (Table 1: int8 vectors, d = 100) with the
subspace counts M in {20, 25, 50} (5, 4 and 2 coordinates; the scans run 32
or 64 subspaces, the extra ones with code 0 and zero table entries) and the
inner-product metric (-<q, x>, smallest first), against the FP64 oracle run
with the same metric on the same index."""
import numpy as np
import pytest

import oracle
import synth
from parity_checks import (_adc_ref, _batched_adc_bound, _check_bounded_topn, _check_topk, _l2_ref,
                           _lowp_adc_bound)

pytestmark = pytest.mark.gpu

MET = {"L2": oracle.L2, "IP": oracle.IP}


@pytest.fixture(scope="module")
def fa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_16576_b300 as m
    return m


_CACHE = {}


def _index(fa, M, metric, raw=None):
    key = (M, metric, raw)
    if key not in _CACHE:
        mix = synth.spacev_like(1_000_000, M).mix
        base = mix.base(30_000)
        q = mix.queries(24)
        loc = {None: fa.FA_RAW_NONE, "dev": fa.FA_RAW_DEVICE, "host": fa.FA_RAW_HOST_PINNED}[raw]
        ix = fa.fa_build_index(base, fa.build_params(nlist=64, M=M, kmeans_iters=6, raw_location=loc,
                                                     metric=getattr(fa, "FA_METRIC_" + metric)))
        parts = ix.parts()
        off, ids = oracle.lists_from_parts(parts["primary"], parts["rep_off"], parts["rep_ids"],
                                           parts["nlist"])
        _CACHE[key] = dict(base=base, q=q, ix=ix, parts=parts, off=off, ids=ids, metric=MET[metric])
    return _CACHE[key]


@pytest.mark.parametrize("metric", ["L2", "IP"])
@pytest.mark.parametrize("M", [20, 25, 50])
def test_int8_subspace_counts_match_oracle(fa, M, metric):
    """Plain FP32 form (FP32 table built in the scan) with the oracle's probe
    lists: top-10 and top-600 equal the oracle's up to boundary near-ties,
    every distance recomputed by the oracle with the index's metric."""
    s = _index(fa, M, metric)
    assert s["parts"]["M"] == M and s["parts"]["metric"] == (1 if metric == "IP" else 0)
    probes = oracle.coarse(s["q"], s["parts"]["centroids"], 12, metric=s["metric"])
    for k in (10, 600):
        gi, gd = fa.fa_search_ex(s["ix"], s["q"], k, 12, probes=probes)
        oi, od = oracle.search(s["q"], s["parts"]["centroids"], s["parts"]["codebooks"],
                               s["parts"]["codes"], s["off"], s["ids"], 12, k + 1, probes=probes,
                               metric=s["metric"])
        for i in range(s["q"].shape[0]):
            _check_topk(gi[i], gd[i], oi[i, :k], od[i, :k], od[i, k], k, what="k%d q%d" % (k, i),
                        ref_of=_adc_ref(s["q"][i], s["parts"]))


@pytest.mark.parametrize("metric", ["L2", "IP"])
def test_int8_coarse_probe_matches_oracle(fa, metric):
    s = _index(fa, 25, metric)
    got = fa.fa_debug_probes(s["ix"], s["q"], 12)
    ref, d2 = oracle.coarse(s["q"], s["parts"]["centroids"], 13, with_d2=True, metric=s["metric"])
    for i in range(s["q"].shape[0]):
        if got[i].tolist() != ref[i, :12].tolist():
            assert abs(d2[i, 12] - d2[i, 11]) <= 1e-5 * max(abs(d2[i, 11]), 1.0), i


@pytest.mark.parametrize("metric", ["L2", "IP"])
@pytest.mark.parametrize("M", [25, 50])
def test_int8_tensor_core_fp16_within_bound(fa, M, metric):
    """BF16 tensor-core probe and LUT, FP16 table (per-query scan) and the
    batched form (FP16 and FP8): every distance within the table's error bound
    of the oracle's ADC of that id (d / M = 4 or 2, which the tensor-core
    table needs)."""
    s = _index(fa, M, metric)
    tc = fa.FA_GEMM_BF16_TC
    probes = oracle.coarse(s["q"], s["parts"]["centroids"], 12, metric=s["metric"])
    oi, _ = oracle.search(s["q"], s["parts"]["centroids"], s["parts"]["codebooks"], s["parts"]["codes"],
                          s["off"], s["ids"], 12, 50, probes=probes, metric=s["metric"])
    p = fa.search_params(lut_prec=fa.FA_LUT_F16, lut_gemm=tc, probe_gemm=tc)
    gi, gd = fa.fa_search_ex(s["ix"], s["q"], 50, 12, p, probes=probes)
    for i in range(s["q"].shape[0]):
        _check_bounded_topn(gi[i], gd[i], oi[i], _adc_ref(s["q"][i], s["parts"]),
                            _lowp_adc_bound(s["q"][i], s["parts"], "F16", True), what=str(i))
    for prec in ("F16", "FP8"):
        p = fa.search_params(lut_prec=getattr(fa, "FA_LUT_" + prec), lut_gemm=tc, flags=fa.FA_BATCHED)
        gi, gd = fa.fa_search_ex(s["ix"], s["q"], 50, 12, p, probes=probes)
        for i in range(s["q"].shape[0]):
            _check_bounded_topn(gi[i], gd[i], oi[i], _adc_ref(s["q"][i], s["parts"]),
                                _batched_adc_bound(s["q"][i], s["parts"], True, prec), what=prec + str(i))


@pytest.mark.parametrize("raw", ["dev", "host"])
@pytest.mark.parametrize("metric", ["L2", "IP"])
def test_int8_rerank_matches_oracle(fa, metric, raw):
    """Algorithm 1 over int8 raw rows (HBM or pinned host memory): the
    oracle's Algorithm 1 with the metric, on the GPU's own ADC top-n, gives
    the GPU's ids and distances (exact: integral queries and int8 rows)."""
    s = _index(fa, 25, metric, raw)
    k, n = 10, 300
    probes = oracle.coarse(s["q"], s["parts"]["centroids"], 12, metric=s["metric"])
    for eps, beta in ((-1.0, 1), (0.0, 2)):
        p = fa.search_params(rerank_n=n, rerank_eps=eps, rerank_beta=beta)
        gi, gd = fa.fa_search_ex(s["ix"], s["q"], k, 12, p, probes=probes)
        an_i, an_d = fa.fa_search_ex(s["ix"], s["q"], n, 12, probes=probes)
        for i in range(s["q"].shape[0]):
            tasks = an_i[i][an_i[i] >= 0]
            if eps >= 0 and len(np.unique(an_d[i][:len(tasks)])) != len(tasks):
                continue
            oi, od, _ = oracle.rerank(s["q"][i], s["parts"]["raw"], tasks, k, batch=32, eps=eps,
                                      beta=beta, metric=s["metric"])
            assert gi[i].tolist() == oi.tolist(), (eps, i)
            assert gd[i].tolist() == od.astype(np.float32).tolist(), (eps, i)


@pytest.mark.parametrize("M", [20, 25, 50])
def test_identity_codebook_ip_full_probe_is_brute_force(fa, M):
    """int8 vectors that are their own PQ centroids, every list probed, inner
    product: the GPU's IVF-PQ top-k is brute force by -<q, x> (pins the
    padding subspaces, the IP table and the scan together)."""
    rng = np.random.default_rng(400 + M)
    d, n, nlist = 100, 200, 6
    x = rng.integers(-128, 128, size=(n, d)).astype(np.int8)
    dsub = d // M
    cb = np.zeros((M, 256, dsub), np.float32)
    for m in range(M):
        cb[m, :n] = x[:, m * dsub:(m + 1) * dsub]
    codes = np.repeat(np.arange(n, dtype=np.uint8)[:, None], M, axis=1)
    primary = rng.integers(0, nlist, size=n).astype(np.int32)
    cent = rng.normal(size=(nlist, d)).astype(np.float32)
    ix = fa.fa_index_from_parts(cent, cb, codes, primary, metric=fa.FA_METRIC_IP)
    q = rng.integers(-128, 128, size=(9, d)).astype(np.float32)
    gi, gd = fa.fa_search(ix, q, 10, nlist)
    ti, td = oracle.knn(q, x, 11, metric=oracle.IP)
    for i in range(q.shape[0]):
        _check_topk(gi[i], gd[i], ti[i, :10], td[i, :10], td[i, 10], 10, what=str(i),
                    ref_of=_l2_ref(q[i], x, oracle.IP))
