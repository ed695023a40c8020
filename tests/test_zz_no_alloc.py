"""The allocation-free coarse probe (fa_coarse_probe_noalloc).

It exists for callers that cannot allocate device memory: a process whose
device memory belongs to another allocator or a fixed budget, or latency-bound
code that cannot afford a cudaMalloc in the middle of its work. Its scratch is
a fixed array inside the library shared by every call.

The test compares it with the library's regular coarse probe (fa_debug_probes,
which works in a per-index workspace) on two calls in a row, so contents the
shared array keeps from one call cannot leak into the next. Probe lists are
integers and both paths run the same kernels: they must be equal. This file is
collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_16576_b300 as m
    return m


def _index(fa, rng, nlist, d, M=8, n=2000):
    cent = (rng.normal(size=(nlist, d)) * 3).astype(np.float32)
    cb = rng.normal(size=(M, 256, d // M)).astype(np.float32)
    codes = rng.integers(0, 256, size=(n, M)).astype(np.uint8)
    primary = rng.integers(0, nlist, size=n).astype(np.int32)
    return cent, fa.fa_index_from_parts(cent, cb, codes, primary)


# (300000 lists leave 13 query rows per scratch block: 40 queries take 4 blocks)
@pytest.mark.parametrize("nlist,nq,nprobe", [(1000, 300, 16), (300_000, 40, 8)])
def test_noalloc_probe_equals_regular_probe_twice(fa, nlist, nq, nprobe):
    import torch
    rng = np.random.default_rng(nlist)
    d = 32
    cent, ix = _index(fa, rng, nlist, d)
    q = (rng.normal(size=(nq, d)) * 3).astype(np.float32)
    ref = fa.fa_debug_probes(ix, q, nprobe)
    qd = torch.as_tensor(q, device="cuda")
    cd = torch.as_tensor(cent, device="cuda")
    out = torch.empty((nq, nprobe), dtype=torch.int32, device="cuda")
    for _ in range(2):
        out.fill_(-7)
        fa.fa_coarse_probe_noalloc(qd, cd, nprobe, out=out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref)


def test_noalloc_probe_rejects_oversized_and_bad_arguments(fa):
    import torch
    q = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
    c = torch.zeros((16, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(fa.FaError) as e:  # rejected on the host before any launch
        fa.fa_coarse_probe_noalloc(q, c, 4, nlist=(4 << 20) + 1)
    assert e.value.status == fa.FA_ERR_ARG and "capacity" in str(e.value)
    with pytest.raises(fa.FaError) as e:
        fa.fa_coarse_probe_noalloc(q, c, 17)
    assert e.value.status == fa.FA_ERR_ARG
    out = fa.fa_coarse_probe_noalloc(q[:0], c, 4)
    assert out.shape == (0, 4)


def test_noalloc_probe_single_list_many_queries(fa):
    """One list and more query rows than one grid of distance tiles spans in
    y (4194240 rows): the probe runs in row blocks and every query gets list 0."""
    import torch
    nq, d = (4 << 20) + 77, 4
    q = torch.ones((nq, d), dtype=torch.float32, device="cuda")
    c = torch.zeros((1, d), dtype=torch.float32, device="cuda")
    out = torch.full((nq, 1), -7, dtype=torch.int32, device="cuda")
    for _ in range(2):
        fa.fa_coarse_probe_noalloc(q, c, 1, out=out)
        torch.cuda.synchronize()
        assert int((out != 0).sum().item()) == 0
