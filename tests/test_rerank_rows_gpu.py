"""Re-rank row forms against the oracle's Algorithm 1.

uint8 rows are read in 32-byte pieces when a row is a multiple of 32 bytes
(four lanes a row, one 256-bit load for eight rows) and in 16-byte pieces
otherwise. d = 48 takes the 16-byte form, d = 96 the 32-byte form with one
of the four lanes of a row idle (three pieces), d = 256 the 32-byte form over
two rounds of pieces. Each is checked inside the selecting scan (exhaustive,
top-n above 256), in the separate re-rank kernel over the queries handed
back (threshold forced low) and in the separate kernel with Algorithm 1's
early stop (eps 0): integral queries take the exact integer form (the
oracle's distances exactly), shifted queries the float form. The FP16 table
is built by the CUDA-core kernel (these shapes are outside the tensor-core
table's d <= 128 with d / M dividing 16)."""
import numpy as np
import pytest

import oracle
import synth
from parity_checks import _check_topk, _l2_ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_16576_b300 as m
    return m


_IX = {}


def _index(fa, d):
    if d not in _IX:
        mix = synth.Mixture(d, 12, 8.0, kind="u8", seed=d)
        base = mix.base(20_000)
        q = mix.queries(8)
        M = 16 if d == 48 else 32
        ix = fa.fa_build_index(base, fa.build_params(nlist=32, M=M, kmeans_iters=4,
                                                     raw_location=fa.FA_RAW_DEVICE))
        _IX[d] = dict(q=q, ix=ix, parts=ix.parts())
    return _IX[d]


@pytest.mark.parametrize("d", [48, 96, 256])
@pytest.mark.parametrize("mode", ["fused", "handed_back", "early_stop"])
@pytest.mark.parametrize("shift", [0.0, 0.3])
def test_rerank_row_forms(fa, d, mode, shift):
    s = _index(fa, d)
    k, npb, n = 10, 12, 300
    q = (s["q"] + np.float32(shift)).astype(np.float32)
    probes = oracle.coarse(q, s["parts"]["centroids"], npb)
    eps, beta = (0.0, 2) if mode == "early_stop" else (-1.0, 1)
    p = fa.search_params(rerank_n=n, rerank_batch=32, rerank_eps=eps, rerank_beta=beta,
                         lut_prec=fa.FA_LUT_F16, lut_gemm=fa.FA_GEMM_SIMT_F32)
    fa.fa_debug_tau_sigma(-1000.0 if mode == "handed_back" else 4.0)
    try:
        gi, gd, st = fa.fa_search_ex(s["ix"], q, k, npb, p, probes=probes, stats=True)
        pa = fa.search_params(lut_prec=fa.FA_LUT_F16, lut_gemm=fa.FA_GEMM_SIMT_F32)
        an_i, _ = fa.fa_search_ex(s["ix"], q, n, npb, pa, probes=probes)
    finally:
        fa.fa_debug_tau_sigma(4.0)
    for i in range(q.shape[0]):
        # the GPU's own ADC top-n, in its order, is Algorithm 1's input
        tasks = an_i[i][an_i[i] >= 0]
        oi, od, nb = oracle.rerank(q[i], s["parts"]["raw"], tasks, k, batch=32, eps=eps, beta=beta)
        if shift == 0.0:
            assert gd[i].tolist() == od.astype(np.float32).tolist(), (d, mode, i)
            assert gi[i].tolist() == oi.tolist(), (d, mode, i)
        else:
            _check_topk(gi[i], gd[i], oi, od, od[-1], k, what="%d %s %d" % (d, mode, i),
                        ref_of=_l2_ref(q[i], s["parts"]["raw"]))
        assert st[i, 2] == nb, (d, mode, i, st[i], nb)
