"""Seeded synthetic inputs for the IVF-PQ filtering path.

This module only draws random numbers and shapes them into base vectors and
queries. It holds none of the search arithmetic (no distances, lookup tables,
clustering or selection), so that both the CPU oracle and the CUDA path can be
fed from it without sharing any code of the method.

Every draw comes from a Philox-4x64 counter-based generator (Salmon et al.,
SC'11) keyed by (seed, stream, chunk of rows). Any chunk-aligned row range can
therefore be regenerated on its own and yields the same rows as a full draw.
Rows are produced in chunks of ``CHUNK`` rows.

The workload shapes follow the paper's billion-scale datasets (Table 1):
SIFT-like d=128 uint8 and DEEP-like d=96 float32 unit-norm data, here drawn
from isotropic Gaussian mixtures because the datasets themselves are not used.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

BASE_SEED = 20240916
# stream ids (the generator key's second word)
STREAM_MEANS = 0
STREAM_BASE = 1
STREAM_QUERIES = 2
STREAM_KMEANS = 3
STREAM_PQ = 4
STREAM_ARRIVALS = 5
STREAM_PARAMS = 6

CHUNK = 4096


def philox(seed: int, stream: int, chunk: int) -> np.random.Generator:
    """A numpy Generator on Philox keyed by (seed, stream, chunk)."""
    key = np.array([seed & 0xFFFFFFFFFFFFFFFF,
                    ((stream & 0xFFFF) << 48) | (chunk & 0xFFFFFFFFFFFF)],
                   dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


def _threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


@dataclass(frozen=True)
class Mixture:
    """Isotropic Gaussian mixture: ``ncomp`` means drawn U[lo, hi]^d,
    per-coordinate std ``sigma``, uniform weights.

    ``kind`` selects the output form:
      * ``"f32"``   plain float32 samples;
      * ``"u8"``    samples clipped to [0, 255] and rounded (SIFT-like);
      * ``"unit"``  float32 samples scaled to unit L2 norm (DEEP-like);
      * ``"i8"``    samples clipped to [-128, 127] and rounded (SPACEV-like).
    """
    d: int
    ncomp: int
    sigma: float = 8.0
    lo: float = 0.0
    hi: float = 100.0
    kind: str = "f32"
    seed: int = BASE_SEED

    def means(self) -> np.ndarray:
        g = philox(self.seed, STREAM_MEANS, 0)
        return g.uniform(self.lo, self.hi, size=(self.ncomp, self.d))

    def _chunk(self, stream: int, c: int, rows: int, means: np.ndarray):
        g = philox(self.seed, stream, c)
        comp = g.integers(0, self.ncomp, size=rows)
        x = g.standard_normal(size=(rows, self.d), dtype=np.float64)
        x *= self.sigma
        x += means[comp]
        if self.kind == "u8":
            np.clip(x, 0.0, 255.0, out=x)
            return np.rint(x).astype(np.uint8)
        if self.kind == "i8":
            np.clip(x, -128.0, 127.0, out=x)
            return np.rint(x).astype(np.int8)
        if self.kind == "unit":
            x /= np.linalg.norm(x, axis=1, keepdims=True)
        return x.astype(np.float32)

    def rows(self, start: int, stop: int, stream: int = STREAM_BASE) -> np.ndarray:
        """Rows [start, stop) of the given stream (chunk-aligned regeneration)."""
        if stop <= start:
            return np.zeros((0, self.d), dtype=self.dtype)
        means = self.means()
        c0, c1 = start // CHUNK, (stop - 1) // CHUNK
        out = np.empty((stop - start, self.d), dtype=self.dtype)

        def work(c):
            lo = c * CHUNK
            blk = self._chunk(stream, c, CHUNK, means)
            a, b = max(lo, start), min(lo + CHUNK, stop)
            out[a - start:b - start] = blk[a - lo:b - lo]

        chunks = range(c0, c1 + 1)
        if len(chunks) > 4:
            with ThreadPoolExecutor(_threads()) as ex:
                list(ex.map(work, chunks))
        else:
            for c in chunks:
                work(c)
        return out

    @property
    def dtype(self):
        return {"u8": np.uint8, "i8": np.int8}.get(self.kind, np.float32)

    def base(self, n: int) -> np.ndarray:
        return self.rows(0, n, STREAM_BASE)

    def queries(self, nq: int, start: int = 0) -> np.ndarray:
        """Queries [start, start + nq) drawn like the base, returned as float32
        (uint8 values are exact in float32)."""
        return self.rows(start, start + nq, STREAM_QUERIES).astype(np.float32)


# ---------------------------------------------------------------------------
# Named workloads (the paper's dataset shapes, Table 1; sizes of the study's
# five configurations).
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Workload:
    name: str
    mix: Mixture
    n: int
    nq: int
    nlist: int
    M: int
    nprobe: int
    k: int


def plain_f32_100k() -> Workload:
    """100k float32 d=128 vectors, 64-component mixture (means U[0,100],
    sigma 8), 256 lists, M=16, 100 queries, nprobe 8, k 10."""
    return Workload("ivfpq-f32-100k-d128-nlist256-M16", Mixture(128, 64, 8.0),
                    100_000, 100, 256, 16, 8, 10)


def sift_like_10m() -> Workload:
    """10M uint8 d=128 vectors (mixture clipped to 0..255 and rounded),
    16384 lists, M=32, 10k queries, nprobe 64, k 10."""
    return Workload("ivfpq-u8-10m-d128-nlist16384-M32", Mixture(128, 64, 8.0, kind="u8"),
                    10_000_000, 10_000, 16384, 32, 64, 10)


def billion_like(n: int = 1_000_000_000) -> Workload:
    """The billion-scale SIFT-like shape: uint8 d=128 vectors from a
    4096-component mixture (clipped to 0..255 and rounded), 262144 lists,
    M=32, 10k queries, nprobe 64 (swept over 64..256), k 10. ``n`` below 1e9
    keeps every other parameter."""
    return Workload("ivfpq-u8-%dm-d128-nlist262144-M32" % (n // 1_000_000),
                    Mixture(128, 4096, 8.0, kind="u8"), n, 10_000, 262144, 32, 64, 10)


def spacev_like(n: int = 10_000_000, M: int = 25) -> Workload:
    """The SPACEV-like shape (Table 1): int8 d=100 vectors from a 64-component
    mixture (means U[-40, 40], sigma 8, clipped to -128..127 and rounded),
    M in {20, 25, 50} subspaces of 5, 4 or 2 coordinates, 16384 lists, 10k
    queries, nprobe 64, k 10."""
    return Workload("ivfpq-i8-%dm-d100-nlist16384-M%d" % (n // 1_000_000, M),
                    Mixture(100, 64, 8.0, lo=-40.0, hi=40.0, kind="i8"), n, 10_000, 16384, M, 64, 10)


def zipf_sizes(nlist: int, n: int, s: float = 1.1) -> np.ndarray:
    """List sizes proportional to i^-s (i = 1..nlist), largest-remainder
    rounding to sum n, each at least 1."""
    w = np.arange(1, nlist + 1, dtype=np.float64) ** (-s)
    w /= w.sum()
    raw = w * (n - nlist)
    base = np.floor(raw).astype(np.int64)
    rem = (n - nlist) - int(base.sum())
    order = np.argsort(-(raw - base), kind="stable")
    base[order[:rem]] += 1
    return base + 1


@dataclass(frozen=True)
class ZipfLists:
    """Unit-norm vectors grouped, by construction, into nlist lists of Zipf(s)
    sizes (DEEP-like d=96 float32). List centres are drawn from an isotropic
    ``ncomp``-component mixture (component means N(0, 1)^d, centre spread
    ``centre_sigma``); a vector is its list's centre plus N(0, sigma^2)
    noise, scaled to unit norm. Rows are ordered by list: row i belongs to the
    list whose size prefix covers i. The normalised centres serve as the IVF
    centroids and ``primary()`` as the assignment (no clustering)."""
    n: int
    d: int = 96
    nlist: int = 65536
    ncomp: int = 1024
    s: float = 1.1
    centre_sigma: float = 0.35
    sigma: float = 0.2
    seed: int = BASE_SEED

    def sizes(self) -> np.ndarray:
        return zipf_sizes(self.nlist, self.n, self.s)

    def _centres_raw(self) -> np.ndarray:
        g = philox(self.seed, STREAM_MEANS, 1)
        means = g.standard_normal(size=(self.ncomp, self.d))
        comp = g.integers(0, self.ncomp, size=self.nlist)
        return means[comp] + self.centre_sigma * g.standard_normal(size=(self.nlist, self.d))

    def centroids(self) -> np.ndarray:
        c = self._centres_raw()
        return (c / np.linalg.norm(c, axis=1, keepdims=True)).astype(np.float32)

    def primary(self) -> np.ndarray:
        return np.repeat(np.arange(self.nlist, dtype=np.int32), self.sizes())

    def _make(self, stream, chunk, lists, centres):
        g = philox(self.seed, stream, chunk)
        x = centres[lists] + self.sigma * g.standard_normal(size=(lists.shape[0], self.d))
        x /= np.linalg.norm(x, axis=1, keepdims=True)
        return x.astype(np.float32)

    def rows(self, start: int, stop: int) -> np.ndarray:
        centres = self._centres_raw()
        bounds = np.concatenate([[0], np.cumsum(self.sizes())])
        out = np.empty((max(0, stop - start), self.d), dtype=np.float32)
        if stop <= start:
            return out
        c0, c1 = start // CHUNK, (stop - 1) // CHUNK

        def work(c):
            lo, hi = c * CHUNK, min((c + 1) * CHUNK, self.n)
            lists = np.searchsorted(bounds, np.arange(lo, hi), side="right") - 1
            blk = self._make(STREAM_BASE, c, lists, centres)
            a, b = max(lo, start), min(hi, stop)
            out[a - start:b - start] = blk[a - lo:b - lo]

        with ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(work, range(c0, c1 + 1)))
        return out

    def base(self) -> np.ndarray:
        return self.rows(0, self.n)

    def queries(self, nq: int) -> np.ndarray:
        """Queries drawn like the base: a uniformly chosen row's list, fresh noise."""
        centres = self._centres_raw()
        bounds = np.concatenate([[0], np.cumsum(self.sizes())])
        g = philox(self.seed, STREAM_QUERIES, 1 << 20)
        lists = np.searchsorted(bounds, g.integers(0, self.n, size=nq), side="right") - 1
        return self._make(STREAM_QUERIES, 1 << 21, lists, centres)


def zipf_unit_100m() -> "ZipfLists":
    """100M unit-norm d=96 vectors, 65536 Zipf(1.1) lists, 1024-component mixture."""
    return ZipfLists(100_000_000)


def poisson_arrivals(rate_qps: float, count: int, seed: int = BASE_SEED) -> np.ndarray:
    """Arrival times (s) of an open-loop Poisson process: exponential gaps."""
    g = philox(seed, STREAM_ARRIVALS, int(rate_qps) & 0xFFFFFFFF)
    return np.cumsum(g.exponential(1.0 / rate_qps, size=count))


def uniform_ints(lo: int, hi: int, count: int, tag: int, seed: int = BASE_SEED) -> np.ndarray:
    """``count`` integers uniform on [lo, hi] (inclusive), stream PARAMS/tag."""
    g = philox(seed, STREAM_PARAMS, tag)
    return g.integers(lo, hi + 1, size=count).astype(np.int32)
