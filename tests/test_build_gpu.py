"""The GPU index build (the offline processing of §3 and the multi-tiered
index of §4.1): PQ encoding on the GPU against a plain nearest-sub-centroid
reference, and the two-level clustering used for many lists, with Eq. 2
boundary replication, at more than a million vectors: the realised
replication, each vector's lists against brute force over all centroids,
and gather + dedup bit-exact against the oracle over the replicated lists."""
import numpy as np
import pytest

import oracle
import synth
from parity_checks import _adc_ref, _check_topk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_16576_b300 as m
    return m


def test_gpu_pq_encoding_is_nearest_subcentroid(fa):
    """Every code is the sub-centroid nearest to the vector's sub-vector (FP64
    reference; a different choice only where the two distances are closer
    than FP32 rounding)."""
    mix = synth.Mixture(128, 16, 8.0, kind="u8")
    base = mix.base(20_000)
    ix = fa.fa_build_index(base, fa.build_params(nlist=32, M=32, kmeans_iters=4, use_gpu=1))
    p = ix.parts()
    cb = p["codebooks"].astype(np.float64)
    M, _, dsub = cb.shape
    x = base.astype(np.float64).reshape(-1, M, dsub)
    diff = 0
    for m in range(M):
        d2 = ((x[:, m, None, :] - cb[None, m]) ** 2).sum(-1)  # [n][256]
        best = d2.argmin(1)
        got = p["codes"][:, m].astype(np.int64)
        bad = np.nonzero(got != best)[0]
        if bad.size:
            gd = d2[bad, got[bad]]
            bd = d2[bad, best[bad]]
            assert np.all(gd - bd <= 1e-5 * np.maximum(bd, 1.0)), m
        diff += bad.size
    assert diff <= 1e-4 * base.shape[0] * M


@pytest.fixture(scope="module")
def big(fa):
    """1.2M float vectors d=32 in 32768 lists (two-level clustering), Eq. 2
    replication at 1.08 lists per vector (up to 4 lists)."""
    mix = synth.Mixture(32, 256, 4.0, lo=-20.0, hi=20.0)
    base = mix.base(1_200_000)
    ix = fa.fa_build_index(base, fa.build_params(nlist=32768, M=16, kmeans_iters=4, repl_eps=-1.08,
                                                 max_lists_per_vec=4, use_gpu=1))
    parts = ix.parts()
    off, ids = oracle.lists_from_parts(parts["primary"], parts["rep_off"], parts["rep_ids"],
                                       parts["nlist"])
    return dict(mix=mix, base=base, ix=ix, parts=parts, off=off, ids=ids)


def test_two_level_build_replication_and_lists(fa, big):
    """The realised replication is the requested 1.08 lists per vector; a
    vector's lists are distinct, the primary among them; the primary is the
    nearest list by brute force for nearly every vector (the two-level search
    looks inside the vector's top-level cluster only) and never far from it;
    every replica list is no nearer than the primary."""
    p = big["parts"]
    n = p["n"]
    lpv = (n + p["rep_off"][-1]) / n
    assert 1.06 <= lpv <= 1.10, lpv
    cent = p["centroids"].astype(np.float64)
    rng = np.random.default_rng(5)
    sample = rng.choice(n, size=1500, replace=False)
    lists_of = {}
    rep_off, rep_ids = p["rep_off"], p["rep_ids"]
    owner = np.repeat(np.arange(p["nlist"]), np.diff(rep_off))
    for v, l in zip(rep_ids.tolist(), owner.tolist()):
        lists_of.setdefault(v, []).append(l)
    nearest_hits = 0
    for v in sample.tolist():
        x = big["base"][v].astype(np.float64)
        d2 = ((cent - x) ** 2).sum(1)
        order = np.argsort(d2, kind="stable")
        prim = int(p["primary"][v])
        reps = lists_of.get(v, [])
        assert prim not in reps and len(set(reps)) == len(reps)
        nearest_hits += prim == int(order[0])
        assert d2[prim] <= d2[order[9]] + 1e-6
        for l in reps:
            assert d2[l] >= d2[prim] * (1 - 1e-5)
    assert nearest_hits >= 0.8 * sample.size, nearest_hits


def test_two_level_dedup_bit_exact(fa, big):
    """Gather + dedup over replicated lists of a 1.2M-vector index: the GPU's
    distinct candidates equal the oracle's sort-unique of the probed lists,
    for random probe sets and for the nearest lists of real queries."""
    s = big
    nl = s["parts"]["nlist"]
    rng = np.random.default_rng(11)
    for t in range(12):
        probes = rng.choice(nl, size=int(rng.integers(8, 200)), replace=False).astype(np.int32)
        got = fa.fa_debug_candidates(s["ix"], probes=probes)
        ref, _ = oracle.candidates(probes, s["off"], s["ids"])
        assert got.tolist() == ref.astype(np.int64).tolist(), t
    q = s["mix"].queries(6)
    pr = oracle.coarse(q, s["parts"]["centroids"], 128)
    for i in range(q.shape[0]):
        got = fa.fa_debug_candidates(s["ix"], probes=pr[i])
        ref, gathered = oracle.candidates(pr[i], s["off"], s["ids"])
        assert got.tolist() == ref.astype(np.int64).tolist(), i
        assert gathered > ref.shape[0]  # replicas were gathered and removed


@pytest.mark.parametrize("batched", [False, True])
def test_two_level_search_matches_oracle(fa, big, batched):
    """Top-k over the replicated 1.2M-vector index against the oracle (FP32
    form per query, and the batched FP16 form within its bound)."""
    from parity_checks import _batched_adc_bound, _check_bounded_topn
    s = big
    q = s["mix"].queries(16)
    probes = oracle.coarse(q, s["parts"]["centroids"], 64)
    oi, od = oracle.search(q, s["parts"]["centroids"], s["parts"]["codebooks"], s["parts"]["codes"],
                           s["off"], s["ids"], 64, 101, probes=probes)
    if not batched:
        gi, gd = fa.fa_search_ex(s["ix"], q, 100, 64, probes=probes)
        for i in range(q.shape[0]):
            _check_topk(gi[i], gd[i], oi[i, :100], od[i, :100], od[i, 100], 100, what=str(i),
                        ref_of=_adc_ref(q[i], s["parts"]))
    else:
        p = fa.search_params(lut_prec=fa.FA_LUT_F16, lut_gemm=fa.FA_GEMM_BF16_TC, flags=fa.FA_BATCHED)
        gi, gd = fa.fa_search_ex(s["ix"], q, 100, 64, p, probes=probes)
        for i in range(q.shape[0]):
            _check_bounded_topn(gi[i], gd[i], oi[i, :100], _adc_ref(q[i], s["parts"]),
                                _batched_adc_bound(q[i], s["parts"], True), what=str(i))
