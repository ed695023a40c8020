"""Parity at the full size of the precision workload, in the launch
configuration bench.py times: 10M uint8 d=128 vectors, 16384 lists, M 32,
10k queries, nprobe 144, the ADC top-12288 re-ranked exhaustively on raw rows
in HBM (the selecting scan with the re-rank fused into it). The oracle checks
a sample of queries one by one; the rest of the batch runs in the same calls,
so the sampled rows come out of the full-size launches.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_checks import RTOL, _adc_ref, _check_topk, _lowp_adc_bound

pytestmark = pytest.mark.gpu

SAMPLE = [0, 1111, 4242, 9999]
RECALL_SAMPLE = np.arange(0, 10_000, 40)  # 250 queries
NPROBE, NTOP = 144, 12288  # the bench's operating point


@pytest.fixture(scope="module")
def full(request):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_16576_b300 as fa
    w = synth.sift_like_10m()
    base = w.mix.base(w.n)
    q = w.mix.queries(w.nq)
    ix = fa.fa_build_index(base, fa.build_params(nlist=w.nlist, M=w.M, kmeans_iters=25,
                                                 raw_location=fa.FA_RAW_DEVICE))
    parts = ix.parts()
    off, ids = oracle.lists_from_parts(parts["primary"], parts["rep_off"], parts["rep_ids"],
                                       parts["nlist"])
    probes = oracle.coarse(q[SAMPLE], parts["centroids"], NPROBE)
    return dict(fa=fa, w=w, base=base, q=q, ix=ix, parts=parts, off=off, ids=ids, probes=probes)


def _batch_probes(s):
    """Probe lists for the whole batch: the GPU's own, with the sampled rows
    replaced by the oracle's exact FP64 ones (so coarse-probe rounding cannot
    leak into the comparison of those rows)."""
    pr = s["fa"].fa_debug_probes(s["ix"], s["q"], NPROBE).astype(np.int32)
    pr[SAMPLE] = s["probes"]
    return np.ascontiguousarray(pr)


def _oracle_topn(s, n):
    return oracle.search(s["q"][SAMPLE], s["parts"]["centroids"], s["parts"]["codebooks"],
                         s["parts"]["codes"], s["off"], s["ids"], NPROBE, n + 1, probes=s["probes"])


def test_fullsize_adc_topn_matches_oracle(full):
    """Plain FP32 form (FP32 LUT in the scan): each sampled row's ADC
    top-12288 equals the oracle's FP64 one except at boundary near-ties, with
    every returned id's distance recomputed by the oracle."""
    s, fa = full, full["fa"]
    n = NTOP
    pr = _batch_probes(s)
    gi, gd = fa.fa_search_ex(s["ix"], s["q"], n, NPROBE, fa.search_params(), probes=pr)
    oi, od = _oracle_topn(s, n)
    for j, i in enumerate(SAMPLE):
        _check_topk(gi[i], gd[i], oi[j, :n], od[j, :n], od[j, n], n, what=str(i),
                    ref_of=_adc_ref(s["q"][i], s["parts"]))


def test_fullsize_lowp_adc_topn_within_lut_bound(full):
    """Precision form's ADC (BF16 tensor-core LUT stored as FP16 with a
    per-(query, subspace) scale and offset): each sampled row's top-12288 has
    distinct ids, ascending keys, and every distance within the table's error
    bound of the oracle's FP64 ADC of that id; every id of the oracle's
    top-12288 it leaves out lies, by that bound, at or beyond its n-th key."""
    s, fa = full, full["fa"]
    n = NTOP
    pr = _batch_probes(s)
    tc = fa.FA_GEMM_BF16_TC
    pa = fa.search_params(lut_prec=fa.FA_LUT_F16, lut_gemm=tc, probe_gemm=tc)
    gi, gd = fa.fa_search_ex(s["ix"], s["q"], n, NPROBE, pa, probes=pr)
    oi, od = _oracle_topn(s, n)
    for j, i in enumerate(SAMPLE):
        ids, g = gi[i], np.asarray(gd[i], np.float64)
        assert np.all(ids >= 0) and len(set(ids.tolist())) == n, i
        keys = list(zip(g.tolist(), ids.tolist()))
        assert keys == sorted(keys), i
        ref = _adc_ref(s["q"][i], s["parts"])
        bnd = _lowp_adc_bound(s["q"][i], s["parts"], "F16", True)
        assert np.all(np.abs(g - ref(ids)) <= bnd(ids)), (i, np.max(np.abs(g - ref(ids)) - bnd(ids)))
        T = g[-1]
        missing = np.array(sorted(set(oi[j, :n].tolist()) - set(ids.tolist())), np.int64)
        if missing.size:
            assert np.all(ref(missing) + bnd(missing) >= T), i


def test_fullsize_recall_within_oracle(full):
    """Recall@10 at the bench's operating point (precision form: tensor-core
    probe and LUT, FP16 table, exhaustive re-rank of the ADC top-12288), the
    whole path on each side with its own probe, on a 250-query subsample of
    the full batch: within 0.005 of the oracle's recall against brute-force
    ground truth (the Recall@10 of the paper's evaluation)."""
    s, fa = full, full["fa"]
    tc = fa.FA_GEMM_BF16_TC
    p = fa.search_params(lut_prec=fa.FA_LUT_F16, lut_gemm=tc, probe_gemm=tc, rerank_n=NTOP,
                         rerank_batch=32, rerank_eps=-1.0, rerank_beta=1)
    gi, _ = fa.fa_search_ex(s["ix"], s["q"], 10, NPROBE, p)
    qs = s["q"][RECALL_SAMPLE]
    oi, _ = oracle.search(qs, s["parts"]["centroids"], s["parts"]["codebooks"], s["parts"]["codes"],
                          s["off"], s["ids"], NPROBE, 10, raw=s["parts"]["raw"], rerank_n=NTOP,
                          batch=32, eps=-1.0, beta=1)
    ti, td = oracle.knn(qs, s["base"], 10)
    r_gpu = oracle.recall_at(gi[RECALL_SAMPLE], ti, td, at=10)
    r_ora = oracle.recall_at(oi, ti, td, at=10)
    assert abs(r_gpu - r_ora) <= 0.005, (r_gpu, r_ora)
    assert r_ora >= 0.85, r_ora


def test_fullsize_recall_point_matches_oracle(full):
    """Precision form at the bench's operating point (BF16 tensor-core probe
    and LUT, FP16 LUT, exhaustive re-rank of the ADC top-12288 fused into the
    scan): each sampled row equals the oracle's Algorithm 1 applied to the
    GPU's own ADC top-12288 (checked above for the FP32 form), bit for bit
    (uint8 data and integral queries: exact distances are integers), with
    every one of the 12288 handed to the re-rank."""
    s, fa = full, full["fa"]
    n = NTOP
    pr = _batch_probes(s)
    tc = fa.FA_GEMM_BF16_TC
    p = fa.search_params(lut_prec=fa.FA_LUT_F16, lut_gemm=tc, probe_gemm=tc, rerank_n=n,
                         rerank_batch=32, rerank_eps=-1.0, rerank_beta=1)
    gi, gd, st = fa.fa_search_ex(s["ix"], s["q"], 10, NPROBE, p, probes=pr, stats=True)
    pa = fa.search_params(lut_prec=fa.FA_LUT_F16, lut_gemm=tc, probe_gemm=tc)
    an_i, _ = fa.fa_search_ex(s["ix"], s["q"], n, NPROBE, pa, probes=pr)
    raw = s["parts"]["raw"]
    for i in SAMPLE:
        tasks = an_i[i][an_i[i] >= 0]
        assert len(tasks) == n
        oi, od, nb = oracle.rerank(s["q"][i], raw, tasks, 10, batch=32, eps=-1.0, beta=1)
        assert gi[i].tolist() == oi.tolist(), i
        assert gd[i].tolist() == od.astype(np.float32).tolist(), i
        assert st[i, 3] == n and st[i, 2] == nb == n // 32, (i, st[i])
