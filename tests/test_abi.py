"""The C-ABI library loads and exports every entry point include/fa.h
declares, its structs have the layout the Python binding assumes, and calls
fail with status codes (never a crash) where no GPU is present. No compute
call runs here."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import paper_2409_16576_b300 as fa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fa.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fa_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert len(names) >= 17
    out = subprocess.run(["nm", "-D", "--defined-only", fa.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fa_[a-z_0-9]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert sorted(fa.EXPORTS) == names


def test_struct_layouts_match_header():
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "fa.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(fa_build_params), sizeof(fa_index_parts),
         sizeof(fa_search_params), sizeof(fa_index_info));
  printf("%zu %zu %zu %zu %zu %zu %zu\n", offsetof(fa_search_params, stats), offsetof(fa_index_parts, raw),
         offsetof(fa_build_params, use_gpu), offsetof(fa_build_params, metric),
         offsetof(fa_index_parts, metric), offsetof(fa_search_params, page_reads),
         offsetof(fa_search_params, graph_max_check));
  return 0; }
'''
    with tempfile.TemporaryDirectory() as t:
        c = os.path.join(t, "p.c")
        open(c, "w").write(prog)
        exe = os.path.join(t, "p")
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = [int(x) for x in lines[0].split()]
    offs = [int(x) for x in lines[1].split()]
    assert sizes == [C.sizeof(fa.fa_build_params), C.sizeof(fa.fa_index_parts),
                     C.sizeof(fa.fa_search_params), C.sizeof(fa.fa_index_info)]
    assert offs == [fa.fa_search_params.stats.offset, fa.fa_index_parts.raw.offset,
                    fa.fa_build_params.use_gpu.offset, fa.fa_build_params.metric.offset,
                    fa.fa_index_parts.metric.offset, fa.fa_search_params.page_reads.offset,
                    fa.fa_search_params.graph_max_check.offset]


def test_status_strings_and_version():
    assert fa.fa_status_str(fa.FA_OK) == "FA_OK"
    assert fa.fa_status_str(fa.FA_ERR_OVERFLOW) == "FA_ERR_OVERFLOW"
    assert fa.fa_status_str(99) == "FA_ERR_UNKNOWN"
    assert "sm_103a" in fa.fa_version()


def test_defaults():
    p = fa.build_params()
    assert (p.nlist, p.M, p.max_lists_per_vec, p.seed, p.use_gpu) == (256, 16, 1, 20240916, 1)
    s = fa.search_params()
    assert (s.lut_prec, s.rerank_n, s.rerank_batch, s.rerank_beta) == (fa.FA_LUT_F32, 0, 32, 2)


def _parts(M=16, d=32, nlist=4, n=20):
    return (np.zeros((nlist, d), np.float32), np.zeros((M, 256, d // M), np.float32),
            np.zeros((n, M), np.uint8), np.arange(n, dtype=np.int32) % nlist)


@pytest.mark.parametrize("bad", ["M", "primary", "dup", "self"])
def test_parts_validation_rejects_bad_descriptions(bad):
    cent, cb, codes, prim = _parts()
    ro = ri = None
    if bad == "M":  # more subspaces than the widest scan (64)
        cb, codes = np.zeros((80, 256, 2), np.float32), np.zeros((20, 80), np.uint8)
        cent = np.zeros((4, 160), np.float32)
    elif bad == "primary":
        prim = prim.copy()
        prim[3] = 7
    elif bad == "dup":
        ro, ri = np.array([0, 2, 2, 2, 2]), np.array([1, 1])
    elif bad == "self":
        ro, ri = np.array([0, 1, 1, 1, 1]), np.array([4])  # vector 4 has primary list 0
    with pytest.raises(fa.FaError) as e:
        fa.fa_index_from_parts(cent, cb, codes, prim, ro, ri)
    assert e.value.status == fa.FA_ERR_ARG


def test_no_device_is_a_status_not_a_crash():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    cent, cb, codes, prim = _parts()
    with pytest.raises(fa.FaError) as e:
        fa.fa_index_from_parts(cent, cb, codes, prim)
    assert e.value.status == fa.FA_ERR_NODEV


def test_load_rejects_missing_and_foreign_files(tmp_path):
    with pytest.raises(fa.FaError) as e:
        fa.fa_load_index(str(tmp_path / "none.idx"))
    assert e.value.status == fa.FA_ERR_IO
    p = tmp_path / "bad.idx"
    p.write_bytes(b"NOTANIDX" + b"\0" * 64)
    with pytest.raises(fa.FaError) as e:
        fa.fa_load_index(str(p))
    assert e.value.status == fa.FA_ERR_IO


def test_failure_hooks_without_a_device():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    fa.fa_debug_fail_alloc(0)
    with pytest.raises(fa.FaError) as e:
        fa.fa_debug_fail_alloc(-1)
    assert e.value.status == fa.FA_ERR_ARG
    with pytest.raises(fa.FaError) as e:
        fa.fa_debug_timeout(16)
    assert e.value.status == fa.FA_ERR_NODEV
