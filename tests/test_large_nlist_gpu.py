"""Replica dedup beyond 65536 lists.

Above 65536 lists the scans keep a query's probed lists in a small
open-addressing table instead of an nlist-bit bitmap (which at 262144 lists
would take 32 KB of every CTA's shared memory). An index of 70000 lists with
Eq. 2-style replicas (each replicated vector in up to three extra lists)
checks that path against the oracle: every query's gathered and distinct
candidate counts (the scan's own, from its stats) equal the oracle's
gather and sort-unique dedup, and the top-k equals the oracle's, for the
warp top-n scan (k 10) and the CTA-wide selecting scan (k 1000)."""
import numpy as np
import pytest

import oracle
from parity_checks import _adc_ref, _check_topk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_16576_b300 as m
    return m


@pytest.fixture(scope="module")
def big(fa):
    rng = np.random.default_rng(70000)
    nlist, n, d, M = 70000, 400_000, 16, 8
    cent = rng.normal(size=(nlist, d)).astype(np.float32)
    cb = rng.normal(size=(M, 256, d // M)).astype(np.float32)
    codes = rng.integers(0, 256, size=(n, M)).astype(np.uint8)
    primary = rng.integers(0, nlist, size=n).astype(np.int32)
    # replicas: 30 % of the vectors in 1..3 further distinct lists
    reps = [[] for _ in range(nlist)]
    for v in np.nonzero(rng.random(n) < 0.3)[0]:
        extra = rng.choice(nlist, size=int(rng.integers(1, 4)) + 1, replace=False)
        for l in [int(x) for x in extra if x != primary[v]][:3]:
            reps[l].append(int(v))
    rep_off = np.zeros(nlist + 1, np.int64)
    rep_off[1:] = np.cumsum([len(r) for r in reps])
    rep_ids = np.array([v for r in reps for v in r], np.int64)
    ix = fa.fa_index_from_parts(cent, cb, codes, primary, rep_off, rep_ids)
    parts = ix.parts()
    off, ids = oracle.lists_from_parts(parts["primary"], parts["rep_off"], parts["rep_ids"], nlist)
    q = rng.normal(size=(24, d)).astype(np.float32)
    return dict(ix=ix, parts=parts, off=off, ids=ids, q=q, nlist=nlist)


@pytest.mark.parametrize("k", [10, 1000])
def test_large_nlist_dedup_counts_and_topk(fa, big, k):
    s = big
    rng = np.random.default_rng(k)
    npb = 300  # ~1700 primaries and ~1500 replica entries per query
    probes = np.stack([rng.choice(s["nlist"], size=npb, replace=False) for _ in range(s["q"].shape[0])])
    probes = probes.astype(np.int32)
    gi, gd, st = fa.fa_search_ex(s["ix"], s["q"], k, npb, probes=probes, stats=True)
    oi, od = oracle.search(s["q"], s["parts"]["centroids"], s["parts"]["codebooks"], s["parts"]["codes"],
                           s["off"], s["ids"], npb, k + 1, probes=probes)
    for i in range(s["q"].shape[0]):
        ref, gathered = oracle.candidates(probes[i], s["off"], s["ids"])
        assert st[i, 0] == gathered and st[i, 1] == ref.shape[0], (i, st[i], gathered, ref.shape[0])
        _check_topk(gi[i], gd[i], oi[i, :k], od[i, :k], od[i, k], k, what=str(i),
                    ref_of=_adc_ref(s["q"][i], s["parts"]))
