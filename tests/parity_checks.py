"""Checks shared by the parity tests: every expected value comes from the
FP64 oracle (recomputed per id, never taken from the GPU), and the bounds are
derived from the arithmetic each form does."""
import numpy as np

import oracle

RTOL = 1e-4


def _adc_ref(q, parts):
    """The oracle's FP64 ADC distance (Eq. 1) of given vector ids for query q:
    its own table over the index's codebooks, summed over the ids' codes."""
    t = oracle.lut(q, parts["codebooks"])
    return lambda ids: oracle.adc(t, parts["codes"], np.asarray(ids, np.int64).astype(np.uint32))


def _l2_ref(q, raw):
    """The oracle's FP64 exact squared L2 of given vector ids (the re-rank's
    distances, Algorithm 1)."""
    return lambda ids: oracle.exact_l2(q, raw, np.asarray(ids, np.int64))


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


def _lowp_lut_bound(q, cb, prec, tc):
    """Per-entry bound [M][256] on |table entry - FP64 value| of an FP16 / FP8
    table with a per-(query, subspace) scale and offset: half an ulp of the
    stored residual (relative), an FP32 rounding margin, the FP8 subnormal
    step, and the tensor-core form's rounding when the table comes from the
    BF16 GEMM (hi/lo split: 4e-5 of the expanded form's terms)."""
    rel = 2.0 ** -11 if prec == "F16" else 2.0 ** -4
    ref = oracle.lut(q, cb)
    resid = ref - ref.min(axis=1, keepdims=True)
    scale = resid.max(axis=1, keepdims=True) / (65504.0 if prec == "F16" else 448.0)
    bound = resid * rel + 1e-5 * np.abs(ref) + scale * (2.0 ** -9 if prec == "FP8" else 2.0 ** -24) + 1e-3
    if tc:
        bound = bound + 4e-5 * _expanded_magnitude(q, cb) * (1 + rel)
    return bound


def _lowp_adc_bound(q, parts, prec, tc):
    """ids -> bound on |low-precision ADC - FP64 ADC|: the sum of the entry
    bounds the ids' codes pick, plus FP32 summation (2e-6 relative)."""
    b = _lowp_lut_bound(q, parts["codebooks"], prec, tc)
    t = oracle.lut(q, parts["codebooks"])

    def f(ids):
        u = np.asarray(ids, np.int64).astype(np.uint32)
        return oracle.adc(b, parts["codes"], u) + 2e-6 * oracle.adc(t, parts["codes"], u) + 1e-3
    return f
