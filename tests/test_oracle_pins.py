"""Pins of the FP64 oracle against things other than itself: values worked by
hand from the paper's definitions (tests/golden), library routines (scipy's
cdist, numpy's lexsort, Python sets), closed forms and invariants.

Each test names the step of the paper it pins. None needs a GPU.
"""
import json
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle


def _rng(seed):
    return np.random.default_rng(seed)


def _lex_topk(dist_row, k):
    ids = np.arange(dist_row.shape[0])
    order = np.lexsort((ids, dist_row))
    return order[:k], dist_row[order[:k]]


# ---------------------------------------------------------------------------
# Eq. 1: LUT and ADC
# ---------------------------------------------------------------------------

def test_lut_adc_golden(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "lut_adc_toy.json")))
    M = g["M"]
    q = np.array(g["query"], dtype=np.float32)
    dsub = q.shape[0] // M
    cb = np.zeros((M, 256, dsub), dtype=np.float32)
    for m, ents in g["centroids"].items():
        for c, v in ents.items():
            cb[int(m), int(c)] = v
    t = oracle.lut(q, cb)
    for m, c, v in g["lut"]:
        assert t[m, c] == v
    codes = np.array(g["codes"], dtype=np.uint8)
    got = oracle.adc(t, codes, np.arange(codes.shape[0]))
    assert got.tolist() == g["adc"]


@pytest.mark.parametrize("d,M", [(16, 4), (128, 16), (128, 32), (96, 48)])
def test_lut_matches_cdist_per_subspace(d, M):
    r = _rng(d * 100 + M)
    dsub = d // M
    q = r.normal(size=d).astype(np.float32) * 10
    cb = r.normal(size=(M, 256, dsub)).astype(np.float32) * 10
    t = oracle.lut(q, cb)
    for m in range(M):
        ref = cdist(q[m * dsub:(m + 1) * dsub][None].astype(np.float64),
                    cb[m].astype(np.float64), "sqeuclidean")[0]
        np.testing.assert_allclose(t[m], ref, rtol=1e-12, atol=1e-9)


def _identity_index(x, M):
    """Each vector is its own PQ centroid: C_m[i] = x_i's m-th sub-vector and
    code[i][m] = i (n <= 256)."""
    n, d = x.shape
    dsub = d // M
    cb = np.zeros((M, 256, dsub), dtype=np.float32)
    for m in range(M):
        cb[m, :n] = x[:, m * dsub:(m + 1) * dsub]
    codes = np.repeat(np.arange(n, dtype=np.uint8)[:, None], M, axis=1)
    return cb, codes


@pytest.mark.parametrize("M", [1, 4, 16, 32])
def test_identity_codebook_adc_is_exact_l2(M):
    r = _rng(7 + M)
    n, d = 200, 64 if M != 32 else 128
    x = r.normal(size=(n, d)).astype(np.float32) * 5
    q = r.normal(size=d).astype(np.float32) * 5
    cb, codes = _identity_index(x, M)
    t = oracle.lut(q, cb)
    got = oracle.adc(t, codes, np.arange(n))
    ref = cdist(q[None].astype(np.float64), x.astype(np.float64), "sqeuclidean")[0]
    np.testing.assert_allclose(got, ref, rtol=1e-12)


def test_adc_uses_code_of_each_subspace():
    """A vector whose codes differ per subspace picks a different centroid in
    each subspace (a transposed code index would read the wrong entries)."""
    r = _rng(3)
    M, dsub = 8, 2
    cb = r.normal(size=(M, 256, dsub)).astype(np.float32)
    q = r.normal(size=M * dsub).astype(np.float32)
    codes = r.integers(0, 256, size=(50, M)).astype(np.uint8)
    t = oracle.lut(q, cb)
    got = oracle.adc(t, codes, np.arange(50))
    # reconstruct each vector from its centroids and take the full distance
    rec = np.stack([np.concatenate([cb[m, codes[v, m]] for m in range(M)]) for v in range(50)])
    ref = cdist(q[None].astype(np.float64), rec.astype(np.float64), "sqeuclidean")[0]
    np.testing.assert_allclose(got, ref, rtol=1e-12)


# ---------------------------------------------------------------------------
# step 2: coarse probe
# ---------------------------------------------------------------------------

def test_coarse_matches_cdist_lexsort():
    r = _rng(11)
    cent = r.normal(size=(300, 32)).astype(np.float32)
    cent[17] = cent[5]  # an exact tie: the smaller list id comes first
    q = r.normal(size=(20, 32)).astype(np.float32)
    q[3] = cent[5]
    probes, d2 = oracle.coarse(q, cent, 12, with_d2=True)
    ref = cdist(q.astype(np.float64), cent.astype(np.float64), "sqeuclidean")
    for i in range(q.shape[0]):
        ids, dd = _lex_topk(ref[i], 12)
        assert probes[i].tolist() == ids.tolist()
        np.testing.assert_allclose(d2[i], dd, rtol=1e-12)
    assert probes[3, 0] == 5 and probes[3, 1] == 17


def test_coarse_self_probe():
    r = _rng(12)
    cent = r.normal(size=(64, 16)).astype(np.float32)
    probes = oracle.coarse(cent, cent, 1)
    assert probes[:, 0].tolist() == list(range(64))


# ---------------------------------------------------------------------------
# steps 3-5: gather and dedup
# ---------------------------------------------------------------------------

def _random_lists(r, n, nlist, rep_frac, max_lists=8):
    primary = r.integers(0, nlist, size=n)
    rep = [[] for _ in range(nlist)]
    nrep = 0
    for v in np.nonzero(r.random(n) < rep_frac)[0]:
        extra = r.choice(nlist, size=min(nlist - 1, r.integers(1, max_lists)), replace=False)
        for l in extra:
            if l != primary[v]:
                rep[l].append(v)
                nrep += 1
    rep_off = np.zeros(nlist + 1, dtype=np.int64)
    rep_off[1:] = np.cumsum([len(a) for a in rep])
    rep_ids = np.array([v for a in rep for v in a], dtype=np.int64)
    return primary, rep_off, rep_ids, nrep


def test_candidates_full_probe_counts():
    r = _rng(21)
    n, nlist = 3000, 40
    primary, rep_off, rep_ids, nrep = _random_lists(r, n, nlist, 0.1)
    off, ids = oracle.lists_from_parts(primary, rep_off, rep_ids, nlist)
    u, gathered = oracle.candidates(np.arange(nlist), off, ids)
    assert gathered == n + nrep
    assert u.shape[0] == n
    assert u.tolist() == list(range(n))


def test_candidates_match_set_union():
    r = _rng(22)
    n, nlist = 5000, 64
    primary, rep_off, rep_ids, _ = _random_lists(r, n, nlist, 0.2)
    off, ids = oracle.lists_from_parts(primary, rep_off, rep_ids, nlist)
    for t in range(10):
        probes = r.choice(nlist, size=r.integers(1, 20), replace=False)
        u, g = oracle.candidates(probes, off, ids)
        ref = set()
        cnt = 0
        for l in probes:
            members = set(np.nonzero(primary == l)[0].tolist())
            members |= set(rep_ids[rep_off[l]:rep_off[l + 1]].tolist())
            cnt += (primary == l).sum() + rep_off[l + 1] - rep_off[l]
            ref |= members
        assert u.tolist() == sorted(ref)
        assert g == cnt


def test_candidates_empty_lists():
    off = np.array([0, 0, 0, 3], dtype=np.int64)
    ids = np.array([7, 2, 7], dtype=np.int64)
    u, g = oracle.candidates([0, 1], off, ids)
    assert u.shape[0] == 0 and g == 0
    u, g = oracle.candidates([2, 0], off, ids)
    assert u.tolist() == [2, 7] and g == 3


# ---------------------------------------------------------------------------
# step 7: top-n
# ---------------------------------------------------------------------------

def test_topn_matches_lexsort_with_ties_and_padding():
    r = _rng(31)
    d = r.integers(0, 20, size=500).astype(np.float64)  # many exact ties
    ids = r.permutation(10_000)[:500].astype(np.uint32)
    oi, od = oracle.topn(d, ids, 37)
    order = np.lexsort((ids.astype(np.int64), d))[:37]
    assert oi.tolist() == ids[order].astype(np.int64).tolist()
    assert od.tolist() == d[order].tolist()
    oi, od = oracle.topn(d[:5], ids[:5], 8)
    assert oi[5:].tolist() == [-1, -1, -1] and np.all(np.isinf(od[5:]))


# ---------------------------------------------------------------------------
# step 8: Algorithm 1 + Eq. 3
# ---------------------------------------------------------------------------

def test_rerank_golden_delta_sequence(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "rerank_toy.json")))
    raw = np.array(g["raw"], dtype=np.float32)[:, None]
    q = np.array(g["query"], dtype=np.float32)
    for case in g["cases"]:
        ids, dist, nb = oracle.rerank(q, raw, g["tasks"], g["k"], g["batch"], case["eps"],
                                      case["beta"])
        assert nb == case["batches"], case
        assert ids.tolist() == case["ids"], case
        assert dist.tolist() == case["dists"], case


@pytest.mark.parametrize("raw_kind", ["u8", "f32"])
def test_rerank_never_stopping_is_exact_topk(raw_kind):
    r = _rng(41)
    n, d, k = 400, 24, 10
    raw = r.integers(0, 256, size=(n, d)).astype(np.uint8) if raw_kind == "u8" else \
        r.normal(size=(n, d)).astype(np.float32)
    q = raw[5].astype(np.float32) + 1
    tasks = r.permutation(n)[:100]
    ids, dist, nb = oracle.rerank(q, raw, tasks, k, 32, eps=-1.0, beta=2)
    assert nb == 4  # ceil(100 / 32), the ragged last batch included
    ref = cdist(q[None].astype(np.float64), raw[tasks].astype(np.float64), "sqeuclidean")[0]
    order = np.lexsort((tasks, ref))[:k]
    assert ids.tolist() == tasks[order].tolist()
    np.testing.assert_allclose(dist, ref[order], rtol=1e-12)


def test_rerank_beta1_eps1_stops_after_first_batch():
    r = _rng(42)
    n, d, k = 300, 16, 10
    raw = r.normal(size=(n, d)).astype(np.float32)
    q = r.normal(size=d).astype(np.float32)
    tasks = r.permutation(n)[:100]
    ids, dist, nb = oracle.rerank(q, raw, tasks, k, 32, eps=1.0, beta=1)
    assert nb == 1
    first = tasks[:32]
    ref = cdist(q[None].astype(np.float64), raw[first].astype(np.float64), "sqeuclidean")[0]
    order = np.lexsort((first, ref))[:k]
    assert ids.tolist() == first[order].tolist()


def test_rerank_padding_and_short_lists():
    raw = np.arange(10, dtype=np.float32)[:, None]
    q = np.zeros(1, dtype=np.float32)
    ids, dist, nb = oracle.rerank(q, raw, [4, 2, -1, -1], 3, 32, eps=-1, beta=1)
    assert ids.tolist() == [2, 4, -1] and nb == 1
    assert dist[:2].tolist() == [4.0, 16.0] and np.isinf(dist[2])
    ids, dist, nb = oracle.rerank(q, raw, [], 3, 32, eps=0, beta=1)
    assert nb == 0 and ids.tolist() == [-1, -1, -1]


# ---------------------------------------------------------------------------
# ground truth and the pipeline
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_knn_matches_cdist(kind):
    r = _rng(51)
    n, d = 2000, 20
    base = r.integers(0, 256, size=(n, d)).astype(np.uint8) if kind == "u8" else \
        r.normal(size=(n, d)).astype(np.float32)
    base[100] = base[10]  # a tie
    q = np.concatenate([base[10:11].astype(np.float32),
                        r.normal(size=(6, d)).astype(np.float32) * 40 + 128])
    ids, dist = oracle.knn(q, base, 15)
    ref = cdist(q.astype(np.float64), base.astype(np.float64), "sqeuclidean")
    for i in range(q.shape[0]):
        o, dd = _lex_topk(ref[i], 15)
        assert ids[i].tolist() == o.tolist()
        np.testing.assert_allclose(dist[i], dd, rtol=1e-12)
    assert ids[0, 0] == 10 and ids[0, 1] == 100


def _identity_ivf(r, n, d, M, nlist, rep_frac):
    x = (r.normal(size=(n, d)) * 6).astype(np.float32)
    cb, codes = _identity_index(x, M)
    cent = r.normal(size=(nlist, d)).astype(np.float32)
    primary, rep_off, rep_ids, _ = _random_lists(r, n, nlist, rep_frac)
    off, ids = oracle.lists_from_parts(primary, rep_off, rep_ids, nlist)
    return x, cb, codes, cent, off, ids


@pytest.mark.parametrize("M", [4, 16])
def test_search_identity_full_probe_equals_knn(M):
    """With every vector its own PQ centroid and every list probed, IVF-PQ
    top-k is exact k-NN (pins gather, dedup, LUT, ADC and top-k together)."""
    r = _rng(61 + M)
    n, d, nlist, k = 240, 32, 12, 10
    x, cb, codes, cent, off, ids = _identity_ivf(r, n, d, M, nlist, 0.3)
    q = (r.normal(size=(15, d)) * 6).astype(np.float32)
    oi, od, st = oracle.search(q, cent, cb, codes, off, ids, nprobe=nlist, k=k, stats=True)
    gi, gd = oracle.knn(q, x, k)
    assert oi.tolist() == gi.tolist()
    np.testing.assert_allclose(od, gd, rtol=1e-10)
    assert np.all(st[:, 1] == n)
    assert np.all(st[:, 0] == off[-1])


def test_search_rerank_identity_equals_knn():
    """Re-ranking never stops (eps < 0) and n covers every vector: the
    result is exact k-NN with exact distances."""
    r = _rng(71)
    n, d, nlist, k = 200, 16, 8, 10
    x, cb, codes, cent, off, ids = _identity_ivf(r, n, d, 4, nlist, 0.0)
    # perturb the codebook so that ADC order differs from exact order
    cb = cb + r.normal(size=cb.shape).astype(np.float32) * 2
    q = (r.normal(size=(9, d)) * 6).astype(np.float32)
    oi, od, st = oracle.search(q, cent, cb, codes, off, ids, nprobe=nlist, k=k, raw=x,
                               rerank_n=n, batch=32, eps=-1.0, beta=1, stats=True)
    gi, gd = oracle.knn(q, x, k)
    assert oi.tolist() == gi.tolist()
    np.testing.assert_allclose(od, gd, rtol=1e-12)
    assert np.all(st[:, 2] == (n + 31) // 32)


def test_search_given_probes_and_fewer_candidates_than_k():
    r = _rng(81)
    n, d, nlist = 60, 8, 10
    x, cb, codes, cent, off, ids = _identity_ivf(r, n, d, 2, nlist, 0.0)
    small = int(np.argmin(np.diff(off)))
    probes = np.full((3, 1), small, dtype=np.int32)
    k = int(off[small + 1] - off[small]) + 4
    oi, od = oracle.search(x[:3], cent, cb, codes, off, ids, nprobe=1, k=k, probes=probes)
    assert np.all(oi[:, -4:] == -1) and np.all(np.isinf(od[:, -4:]))
    members = sorted(ids[off[small]:off[small + 1]].tolist())
    for i in range(3):
        assert sorted(oi[i, :k - 4].tolist()) == members


def test_recall_helper():
    gt = np.array([[1, 2, 3, 4]])
    gd = np.array([[1.0, 2.0, 3.0, 3.0]])
    assert oracle.recall_at(np.array([[1, 2, 9, 8]]), gt, gd, at=4) == 0.5
    # 9 ties the 4th neighbour's distance: counts when exact distances are given
    assert oracle.recall_at(np.array([[1, 2, 9, 8]]), gt, gd,
                            exact_found_dist=np.array([[1.0, 2.0, 3.0, 5.0]]), at=4) == 0.75


# ---------------------------------------------------------------------------
# Inner-product metric and int8 rows (the SPACEV-like workload of Table 1:
# int8 vectors, d = 100, M in {20, 25, 50})
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,M", [(100, 20), (100, 25), (100, 50), (128, 32)])
def test_lut_ip_matches_numpy_dot_per_subspace(d, M):
    """Eq. 1's terms for the inner product: LUT[m][c] = -<q_m, C_m[c]>."""
    rng = _rng(d + M)
    q = rng.normal(size=d).astype(np.float32)
    cb = rng.normal(size=(M, 256, d // M)).astype(np.float32)
    t = oracle.lut(q, cb, metric=oracle.IP)
    ref = -np.einsum("mj,mcj->mc", q.reshape(M, d // M).astype(np.float64), cb.astype(np.float64))
    np.testing.assert_allclose(t, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("M", [20, 25, 50])
def test_identity_codebook_ip_full_probe_equals_brute_force(M):
    """Every vector its own PQ centroid and every list probed: the oracle's
    IVF-PQ top-k by -<q, x> equals brute force by numpy (int8 rows)."""
    rng = _rng(300 + M)
    d, n, nlist = 100, 200, 6
    x = rng.integers(-128, 128, size=(n, d)).astype(np.int8)
    dsub = d // M
    cb = np.zeros((M, 256, dsub), np.float32)
    for m in range(M):
        cb[m, :n] = x[:, m * dsub:(m + 1) * dsub]
    codes = np.repeat(np.arange(n, dtype=np.uint8)[:, None], M, axis=1)
    primary = rng.integers(0, nlist, size=n).astype(np.int32)
    off, ids = oracle.lists_from_parts(primary, np.zeros(nlist + 1, np.int64), np.zeros(0, np.int64), nlist)
    cent = rng.normal(size=(nlist, d)).astype(np.float32)
    q = rng.integers(-128, 128, size=(7, d)).astype(np.float32)
    oi, od = oracle.search(q, cent, cb, codes, off, ids, nlist, 10, metric=oracle.IP)
    for i in range(q.shape[0]):
        ip = -(x.astype(np.float64) @ q[i].astype(np.float64))
        order = np.lexsort((np.arange(n), ip))[:10]
        assert oi[i].tolist() == order.tolist(), i
        np.testing.assert_allclose(od[i], ip[order], rtol=0, atol=1e-9)


@pytest.mark.parametrize("metric", ["L2", "IP"])
def test_knn_int8_matches_numpy(metric):
    rng = _rng(17)
    x = rng.integers(-128, 128, size=(500, 100)).astype(np.int8)
    q = rng.integers(-128, 128, size=(5, 100)).astype(np.float32)
    m = getattr(oracle, metric)
    oi, od = oracle.knn(q, x, 7, metric=m)
    x64, q64 = x.astype(np.float64), q.astype(np.float64)
    for i in range(5):
        dist = ((x64 - q64[i]) ** 2).sum(1) if metric == "L2" else -(x64 @ q64[i])
        order = np.lexsort((np.arange(500), dist))[:7]
        assert oi[i].tolist() == order.tolist()
        np.testing.assert_allclose(od[i], dist[order], rtol=0, atol=1e-9)
        np.testing.assert_allclose(oracle.exact(q[i], x, order, metric=m), dist[order], rtol=0, atol=1e-9)


def test_coarse_ip_matches_numpy_lexsort():
    rng = _rng(23)
    c = rng.normal(size=(300, 100)).astype(np.float32)
    q = rng.normal(size=(9, 100)).astype(np.float32)
    pr, d2 = oracle.coarse(q, c, 12, with_d2=True, metric=oracle.IP)
    for i in range(9):
        ip = -(c.astype(np.float64) @ q[i].astype(np.float64))
        order = np.lexsort((np.arange(300), ip))[:12]
        assert pr[i].tolist() == order.tolist()
        np.testing.assert_allclose(d2[i], ip[order], rtol=0, atol=1e-9)


def test_rerank_ip_never_stopping_is_exact_topk():
    """Algorithm 1 with eps < 0 over int8 rows by -<q, x>: the exact top-k of
    the candidates (numpy)."""
    rng = _rng(31)
    x = rng.integers(-128, 128, size=(300, 100)).astype(np.int8)
    q = rng.integers(-128, 128, size=100).astype(np.float32)
    tasks = rng.permutation(300)[:120].astype(np.int64)
    oi, od, nb = oracle.rerank(q, x, tasks, 10, batch=32, eps=-1.0, beta=1, metric=oracle.IP)
    ip = -(x[tasks].astype(np.float64) @ q.astype(np.float64))
    order = np.lexsort((tasks, ip))[:10]
    assert oi.tolist() == tasks[order].tolist()
    np.testing.assert_allclose(od, ip[order], rtol=0, atol=1e-9)
    assert nb == 4  # ceil(120 / 32) mini-batches


# ---------------------------------------------------------------------------
# §4.3: storage layout and redundancy-aware I/O deduplication
# ---------------------------------------------------------------------------

def test_io_dedup_worked_example(golden_dir):
    """The paper's example: mini-batch 0 merges V2 and V6 into one read of P0
    and reads P2 for V4 (2 I/Os); mini-batch 1 finds P2 in the buffer for V5
    and reads P1 and P3 (2 I/Os)."""
    g = json.load(open(os.path.join(golden_dir, "io_dedup_example.json")))
    page_of = np.full(10, 7, np.int64)
    for v, p in g["page_of"].items():
        page_of[int(v)] = p
    raw = np.arange(40, dtype=np.float32).reshape(10, 4)
    q = np.zeros(4, np.float32)
    for nb_wanted, reads_wanted in ((1, g["pages_read_per_mini_batch"][0]), (2, g["pages_read"])):
        tasks = np.array(g["tasks"][:nb_wanted * g["batch"]], np.int64)
        _, _, nb, reads = oracle.rerank_pages(q, raw, tasks, 2, page_of, batch=g["batch"], eps=-1.0, beta=1)
        assert (nb, reads) == (nb_wanted, reads_wanted)


def test_page_layout_hand_example():
    """Buckets of 40, 20, 10 and 5 vectors, 32 a page: list 0 fills page 0
    and leaves a tail of 8; the tails (20, 10, 8, 5) pair max with min: page 1
    = {20, 5}, page 2 = {10, 8} (8 + 20 would not fit)."""
    prim = np.repeat(np.arange(4), [40, 20, 10, 5]).astype(np.int32)
    page_of, slot_of, npg = oracle.page_layout(prim, 4, 32)
    assert npg == 3
    pages = [sorted(set(page_of[prim == l].tolist())) for l in range(4)]
    assert pages == [[0, 2], [1], [2], [1]]
    # list 0's first 32 vectors (ascending ids) fill page 0 in order
    assert page_of[:32].tolist() == [0] * 32 and slot_of[:32].tolist() == list(range(32))


def test_page_layout_is_a_packing():
    """Random buckets: every vector has one (page, slot), no slot twice, no
    page above its capacity, every bucket's whole pages its own, and no more
    pages than the whole pages plus the tails need (each shared page holds at
    least one tail; a tail never splits)."""
    rng = _rng(41)
    nlist, cap = 50, 32
    sizes = rng.integers(0, 90, size=nlist)
    prim = np.repeat(np.arange(nlist), sizes).astype(np.int32)
    rng.shuffle(prim)
    page_of, slot_of, npg = oracle.page_layout(prim, nlist, cap)
    n = prim.shape[0]
    pairs = set(zip(page_of.tolist(), slot_of.tolist()))
    assert len(pairs) == n and slot_of.min() >= 0 and slot_of.max() < cap
    assert page_of.min() == 0 and page_of.max() == npg - 1
    per_page = np.bincount(page_of, minlength=npg)
    assert per_page.max() <= cap
    whole = int((sizes // cap).sum())
    tails = int((sizes % cap > 0).sum())
    assert -(-n // cap) <= npg <= whole + tails
    for l in range(nlist):  # a bucket's tail sits in one page
        t = sizes[l] % cap
        if t:
            pg = page_of[prim == l]
            vals, cnts = np.unique(pg, return_counts=True)
            assert (cnts == t).sum() >= 1 or t == cap


def test_io_dedup_counts_distinct_new_pages():
    """One mini-batch reads exactly the distinct pages of its tasks; with the
    buffer, a re-rank reads each distinct page once in all; Algorithm 1's
    results do not change."""
    rng = _rng(43)
    raw = rng.integers(0, 256, size=(400, 16)).astype(np.uint8)
    page_of = rng.integers(0, 40, size=400).astype(np.int64)
    q = rng.integers(0, 256, size=16).astype(np.float32)
    tasks = rng.permutation(400)[:96].astype(np.int64)
    oi, od, nb, reads = oracle.rerank_pages(q, raw, tasks, 10, page_of, batch=96, eps=-1.0, beta=1)
    assert nb == 1 and reads == len(set(page_of[tasks].tolist()))
    oi2, od2, nb2, reads2 = oracle.rerank_pages(q, raw, tasks, 10, page_of, batch=16, eps=-1.0, beta=1)
    assert nb2 == 6 and reads2 == reads
    ri, rd, _ = oracle.rerank(q, raw, tasks, 10, batch=16, eps=-1.0, beta=1)
    assert oi2.tolist() == ri.tolist() and np.array_equal(od2, rd)


# ---------------------------------------------------------------------------
# coarse probe by the navigation graph (§3 step 2, §4.1 "In-memory Indices")
# ---------------------------------------------------------------------------

def test_graph_walk_small_golden(golden_dir):
    """Hand-worked walks on a line graph (the beam, the check budget, seeds
    only, the greedy walk, ties met in either order) and on a branching
    graph (which unexpanded vertex goes next)."""
    g = json.load(open(os.path.join(golden_dir, "graph_walk_small.json")))
    for gr in g["graphs"]:
        heads = np.array(gr["positions"], np.float64)[:, None]
        adj = np.array(gr["adj"], np.int32)
        for c in gr["cases"]:
            out, found, checks = oracle.graph_probe(np.array([[c["query"]]], np.float32), heads, adj,
                                                    c["seeds"], c["beam"], c["max_check"], c["nprobe"])
            assert out[0, :found[0]].tolist() == c["lists"], c["why"]
            assert checks[0] == c["checks"], c["why"]


def test_graph_walk_complete_graph_is_exact_probe():
    """Every vertex linked to every other: the first expansion evaluates all
    lists, so the walk returns the exact top-m (pinned above against cdist)
    for any budget that lets the seed be expanded (the budget is checked
    before an expansion, not inside one); a budget of one check stops at
    the seed."""
    rng = np.random.default_rng(61)
    nlist, d, nq, m = 120, 8, 30, 12
    cent = rng.integers(0, 256, size=(nlist, d)).astype(np.float32)
    q = rng.integers(0, 256, size=(nq, d)).astype(np.float32)
    adj = np.array([[u for u in range(nlist) if u != v] for v in range(nlist)], np.int32)
    ref = oracle.coarse(q, cent, m)
    for max_check in (2, 3, nlist):
        out, found, checks = oracle.graph_probe(q, cent.astype(np.float64), adj, [5], 40, max_check, m)
        assert np.array_equal(out, ref) and np.all(found == m)
        assert np.all(checks == nlist)
    out, found, checks = oracle.graph_probe(q, cent.astype(np.float64), adj, [5], 40, 1, m)
    assert np.all(out[:, 0] == 5) and np.all(found == 1) and np.all(checks == 1)


def test_graph_walk_stays_in_the_seeds_component():
    """Two components: a walk seeded in one never returns a list of the
    other, and returns fewer than m lists when its component is smaller."""
    rng = np.random.default_rng(62)
    d = 4
    cent = rng.normal(size=(20, d))
    # component A = 0..4 (a ring), component B = 5..19 (a ring)
    adj = np.full((20, 2), -1, np.int32)
    for lo, hi in ((0, 5), (5, 20)):
        for v in range(lo, hi):
            adj[v] = [lo + (v - lo - 1) % (hi - lo), lo + (v - lo + 1) % (hi - lo)]
    q = rng.normal(size=(10, d)).astype(np.float32)
    out, found, checks = oracle.graph_probe(q, cent, adj, [2], 16, 100, 8)
    assert np.all(found == 5) and np.all(checks == 5)
    assert np.all(np.sort(out[:, :5], axis=1) == np.arange(5)) and np.all(out[:, 5:] == -1)


def test_graph_heads_rounding():
    """Heads are the centroids; for integer vectors rounded to the nearest
    integer (halves to even) and clipped to the type's range."""
    c = np.array([[0.5, 1.5, 2.5, -0.4, 300.2, -128.7, 127.5, 3.49]], np.float32)
    assert oracle.graph_heads(c, np.uint8).tolist() == [[0, 2, 2, 0, 255, 0, 128, 3]]
    assert oracle.graph_heads(c, np.int8).tolist() == [[0, 2, 2, 0, 127, -128, 127, 3]]
    assert oracle.graph_heads(c, np.float32).tolist() == c.astype(np.float64).tolist()


def test_graph_walk_per_query_seeds():
    """Each query's own seeds: the same walk as the query alone with that seed
    list (line graph, hand-worked results), and the nearest-pivot entry is
    numpy's argmin / argsort over the pivots' heads."""
    rng = np.random.default_rng(63)
    heads = np.arange(12, dtype=np.float64)[:, None]
    adj = np.array([[v - 1 if v > 0 else -1, v + 1 if v < 11 else -1] for v in range(12)], np.int32)
    q = np.array([[7.3], [2.2], [10.6]], np.float32)
    seeds = np.array([[0], [11], [4]], np.int32)
    out, found, checks = oracle.graph_probe(q, heads, adj, seeds, 3, 100, 3)
    assert out.tolist() == [[7, 8, 6], [2, 3, 1], [11, 10, 9]]
    for i in range(3):
        o1, f1, c1 = oracle.graph_probe(q[i:i + 1], heads, adj, seeds[i], 3, 100, 3)
        assert o1[0].tolist() == out[i].tolist() and c1[0] == checks[i]
    cent = rng.normal(size=(300, 6))
    pivots = np.arange(0, 300, 7, dtype=np.int32)
    qq = rng.normal(size=(40, 6)).astype(np.float32)
    e = oracle.graph_entry(qq, cent, pivots, 5)
    d2 = ((qq[:, None, :].astype(np.float64) - cent[pivots][None]) ** 2).sum(-1)
    assert np.array_equal(e[:, 0], pivots[np.argmin(d2, axis=1)])
    assert np.array_equal(e, pivots[np.argsort(d2, axis=1, kind="stable")[:, :5]])
