"""Checks shared by the parity tests: every expected value comes from the
FP64 oracle (recomputed per id, never taken from the GPU), and the bounds are
derived from the arithmetic each form does."""
import numpy as np

import oracle

RTOL = 1e-4


def _metric(parts):
    return oracle.IP if parts.get("metric", 0) == 1 else oracle.L2


def _adc_ref(q, parts):
    """The oracle's FP64 ADC distance (Eq. 1) of given vector ids for query q:
    its own table over the index's codebooks (the index's metric), summed
    over the ids' codes."""
    t = oracle.lut(q, parts["codebooks"], metric=_metric(parts))
    return lambda ids: oracle.adc(t, parts["codes"], np.asarray(ids, np.int64).astype(np.uint32))


def _l2_ref(q, raw, metric=None):
    """The oracle's FP64 exact distance of given vector ids (the re-rank's
    distances, Algorithm 1): squared L2, or -<q, x> with metric IP."""
    m = oracle.L2 if metric is None else metric
    return lambda ids: oracle.exact(q, raw, np.asarray(ids, np.int64), metric=m)


def _check_topk(gi, gd, oi, od, o_next, k, rtol=RTOL, what="", ref_of=None):
    """gi/gd: GPU ids/dists of one query; oi/od: oracle's top-k; o_next: the
    oracle's (k+1)-th distance (inf if none); ref_of: ids -> the oracle's own
    FP64 distance of each id (recomputed, never taken from the GPU)."""
    gi = np.asarray(gi)
    gd = np.asarray(gd, dtype=np.float64)
    fin = np.isfinite(od)
    assert np.array_equal(np.isfinite(gd), fin), what
    np.testing.assert_allclose(gd[fin], od[fin], rtol=rtol, atol=1e-3, err_msg=what)
    assert np.all(gi[~fin] == -1), what
    # no id twice in a row
    assert len(set(gi[fin].tolist())) == int(fin.sum()), what
    # every returned id carries the oracle's distance of that id
    if ref_of is not None and fin.any():
        np.testing.assert_allclose(gd[fin], ref_of(gi[fin]), rtol=rtol, atol=1e-3, err_msg=what)
    # ids: equal sets unless the boundary is a near tie
    kth = od[fin][-1] if fin.any() else np.inf
    if set(gi[fin].tolist()) != set(oi[fin].tolist()):
        assert np.isfinite(o_next) and abs(o_next - kth) <= rtol * max(kth, 1.0) + 1e-3, what
        # every id that is not in the oracle's set must sit at the boundary distance
        extra = set(gi[fin].tolist()) - set(oi[fin].tolist())
        for t, x in enumerate(gi):
            if x in extra:
                assert abs(gd[t] - kth) <= rtol * max(kth, 1.0) + 1e-3, what


def _expanded_magnitude(q, cb):
    """|q_m|^2 + |C_m[c]|^2 per entry: the size of the terms the expanded
    (tensor-core) form adds, which bounds its rounding."""
    M, _, dsub = cb.shape
    qn = np.array([(q[m * dsub:(m + 1) * dsub].astype(np.float64) ** 2).sum() for m in range(M)])
    return qn[:, None] + (cb.astype(np.float64) ** 2).sum(2)


def _lowp_lut_bound(q, cb, prec, tc, metric=oracle.L2):
    """Per-entry bound [M][256] on |table entry - FP64 value| of an FP16 / FP8
    table with a per-(query, subspace) scale and offset: half an ulp of the
    stored residual (relative), an FP32 rounding margin, the FP8 subnormal
    step, and the tensor-core form's rounding when the table comes from the
    BF16 GEMM (hi/lo split: 4e-5 of the expanded form's terms)."""
    rel = 2.0 ** -11 if prec == "F16" else 2.0 ** -4
    ref = oracle.lut(q, cb, metric=metric)
    resid = ref - ref.min(axis=1, keepdims=True)
    scale = resid.max(axis=1, keepdims=True) / (65504.0 if prec == "F16" else 448.0)
    bound = resid * rel + 1e-5 * np.abs(ref) + scale * (2.0 ** -9 if prec == "FP8" else 2.0 ** -24) + 1e-3
    if tc:
        bound = bound + 4e-5 * _expanded_magnitude(q, cb) * (1 + rel)
    return bound


def _lowp_adc_bound(q, parts, prec, tc):
    """ids -> bound on |low-precision ADC - FP64 ADC|: the sum of the entry
    bounds the ids' codes pick, plus FP32 summation (2e-6 relative)."""
    b = _lowp_lut_bound(q, parts["codebooks"], prec, tc, _metric(parts))
    t = oracle.lut(q, parts["codebooks"], metric=_metric(parts))

    def f(ids):
        u = np.asarray(ids, np.int64).astype(np.uint32)
        return oracle.adc(b, parts["codes"], u) + 2e-6 * np.abs(oracle.adc(t, parts["codes"], u)) + 1e-3 \
            + 2e-6 * oracle.adc(np.abs(t), parts["codes"], u)
    return f


def _batched_entry_bound(q, parts, tc, prec="F16"):
    """Per-entry bound [M][256] on |entry - FP64 value| of the batched form's
    table, which has one scale per query, at most s_q = 2 (|q|^2 + max
    |C_m[c]|^2) / format max (every entry |q_m - C_m[c]|^2 is below 2 (|q_m|^2
    + |C_m[c]|^2)): half an ulp of the stored residual (2^-11 relative for
    FP16, 2^-4 for FP8 e4m3), the subnormal step below the normal range, an
    FP32 margin, and the tensor-core form's rounding."""
    cb = parts["codebooks"]
    ref = oracle.lut(q, cb, metric=_metric(parts))
    resid = ref - ref.min(axis=1, keepdims=True)
    q64 = np.asarray(q, np.float64)
    fmax, rel, sub = (65504.0, 2.0 ** -11, 2.0 ** -25) if prec == "F16" else (448.0, 2.0 ** -4, 2.0 ** -10)
    sq = 2.0 * ((q64 ** 2).sum() + (cb.astype(np.float64) ** 2).sum(2).max()) / fmax * (1 + 1e-6)
    b = resid * rel + sq * sub + 1e-5 * np.abs(ref) + 1e-3
    if tc:
        b = b + 4e-5 * _expanded_magnitude(q, cb) * (1 + rel)
    return ref, resid, b


def _batched_adc_bound(q, parts, tc, prec="F16"):
    """ids -> bound on |batched-form ADC - FP64 ADC|: the entry bounds the ids'
    codes pick; for FP8, half2 sums over 16 subspaces (15 roundings of 2^-11
    relative to a partial sum of stored residuals); FP32 sums of the entries
    and the offsets, 1e-5 relative."""
    ref, resid, b = _batched_entry_bound(q, parts, tc, prec)

    def f(ids):
        u = np.asarray(ids, np.int64).astype(np.uint32)
        out = oracle.adc(b, parts["codes"], u) + 1e-5 * np.abs(oracle.adc(ref, parts["codes"], u)) + 1e-3
        if prec == "FP8":
            out = out + 15 * 2.0 ** -11 * (1 + 2.0 ** -4) * oracle.adc(resid, parts["codes"], u)
        return out
    return f


def _check_bounded_topn(gi, gd, oi, ref_of, bound_of, what=""):
    """A top-n computed with perturbed distances (each within bound_of(id) of
    the oracle's ref_of(id)): ids distinct, keys ascending, every distance
    within its bound of the oracle's, and every id of the oracle's top-n it
    leaves out at or beyond its n-th key by that bound."""
    gi = np.asarray(gi)
    g = np.asarray(gd, np.float64)
    ok = gi >= 0
    assert np.all(np.isfinite(g[ok])) and np.all(~np.isfinite(g[~ok])), what
    ids = gi[ok]
    assert len(set(ids.tolist())) == ids.size, what
    keys = list(zip(g[ok].tolist(), ids.tolist()))
    assert keys == sorted(keys), what
    r, b = ref_of(ids), bound_of(ids)
    assert np.all(np.abs(g[ok] - r) <= b), (what, float(np.max(np.abs(g[ok] - r) - b)))
    oset = set(int(x) for x in np.asarray(oi) if x >= 0)
    missing = np.array(sorted(oset - set(ids.tolist())), np.int64)
    if missing.size:
        assert ok.all(), what  # a short row must hold every candidate
        T = g[ok][-1]
        assert np.all(ref_of(missing) + bound_of(missing) >= T), what
