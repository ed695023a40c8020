"""Failure detection without faulting the GPU: a device-side wait that runs
out reports FA_ERR_TIMEOUT through the status word and leaves the context
usable; allocation failures injected on the host surface as FA_ERR_OOM at
index upload, workspace growth and server creation, and the next call works."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_16576_b300 as m
    yield m
    m.fa_debug_fail_alloc(0)


def _parts(seed=3):
    mix = synth.Mixture(32, 8, 4.0, lo=-10.0, hi=10.0, seed=seed)
    base = mix.base(3000)
    return base, mix.queries(64)


def test_device_wait_runs_out_and_context_stays_usable(fa):
    base, q = _parts()
    ix = fa.fa_build_index(base, fa.build_params(nlist=16, M=8, kmeans_iters=4))
    before = fa.fa_search_ex(ix, q, 10, 4)
    for polls in (1, 64, 4096):
        with pytest.raises(fa.FaError) as e:
            fa.fa_debug_timeout(polls)
        assert e.value.status == fa.FA_ERR_TIMEOUT
    after = fa.fa_search_ex(ix, q, 10, 4)
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])


def _from_parts(fa, parts):
    return fa.fa_index_from_parts(parts["centroids"], parts["codebooks"], parts["codes"],
                                  parts["primary"], parts["rep_off"], parts["rep_ids"])


@pytest.mark.parametrize("nth", [1, 2, 5])
def test_injected_upload_failure_is_oom_and_the_next_build_works(fa, nth):
    base, q = _parts()
    parts = fa.fa_build_index(base, fa.build_params(nlist=16, M=8, kmeans_iters=4)).parts()
    ix0 = _from_parts(fa, parts)
    fa.fa_debug_fail_alloc(nth)
    with pytest.raises(fa.FaError) as e:
        _from_parts(fa, parts)
    assert e.value.status == fa.FA_ERR_OOM
    ix = _from_parts(fa, parts)
    gi, gd = fa.fa_search_ex(ix, q, 10, 4)
    ri, rd = fa.fa_search_ex(ix0, q, 10, 4)
    assert np.array_equal(gi, ri) and np.array_equal(gd, rd)


def test_injected_workspace_failure_is_oom_and_the_index_stays_usable(fa):
    base, _ = _parts()
    parts = fa.fa_build_index(base, fa.build_params(nlist=16, M=8, kmeans_iters=4)).parts()
    big_q = synth.Mixture(32, 8, 4.0, lo=-10.0, hi=10.0, seed=4).queries(3000)
    twin = _from_parts(fa, parts)
    ri, rd = fa.fa_search_ex(twin, big_q, 10, 4)
    ix = _from_parts(fa, parts)
    si, sd = fa.fa_search_ex(ix, big_q[:8], 10, 4)
    fa.fa_debug_fail_alloc(1)  # the workspace must grow for 3000 queries
    with pytest.raises(fa.FaError) as e:
        fa.fa_search_ex(ix, big_q, 10, 4)
    assert e.value.status == fa.FA_ERR_OOM
    gi, gd = fa.fa_search_ex(ix, big_q, 10, 4)
    assert np.array_equal(gi, ri) and np.array_equal(gd, rd)
    assert np.array_equal(si, ri[:8]) and np.array_equal(sd, rd[:8])


def test_injected_server_slot_failure_is_oom(fa):
    base, q = _parts()
    ix = fa.fa_build_index(base, fa.build_params(nlist=16, M=8, kmeans_iters=4))
    fa.fa_debug_fail_alloc(3)
    with pytest.raises(fa.FaError) as e:
        fa.Server(ix, max_batch=64, slots=2, kmax=10, nprobe_max=16)
    assert e.value.status == fa.FA_ERR_OOM
    srv = fa.Server(ix, max_batch=64, slots=2, kmax=10, nprobe_max=16)
    srv.submit(q[:4], 10, 4)
    got = 0
    for _ in range(200):
        rid, _, _, _, st = srv.poll(max_results=16, timeout_us=20000)
        got += rid.shape[0]
        assert np.all(st == fa.FA_OK)
        if got == 4:
            break
    srv.close()
    assert got == 4
