// Steps 1 and 3-7 of the filtering path for one query per CTA:
//   LUT (step 1)       dist(q_i, c) for the M subspaces, into shared memory
//   gather (3-4)       the probed lists' primary ranges and replica slices
//   dedup (5)          each distinct vector once (probe-set rule below)
//   ADC (6, Eq. 1)     dist(q, v) = sum_i LUT[i][code_i(v)], FP32
//   top-n (7)          variant 1 (n <= 256): per-warp running selection,
//                      merged per CTA; variant 2 (n <= 16384): one CTA per
//                      SM keeps the top-n in shared memory; variant 3 (n <=
//                      16384, rows that may come out unsorted): two CTAs
//                      per SM select below a sampled threshold, and can run
//                      the exhaustive re-rank of step 8 on the result
//
// Layout choices (all made at index upload):
//   * vectors are renumbered so each list's primary members are a contiguous
//     range of internal ids [list_beg[l], list_beg[l+1]);
//   * code rows are rotated: byte s of row v holds the code of subspace
//     (s + v mod 32) mod M. Lane j of a warp scans row v = base + j, so at
//     step s the 32 lanes read 32 different LUT columns p = (v mod 32) + s;
//   * the LUT sits in shared memory as rows of W floats per centroid c with
//     entry p = LUT[p mod M][c] for p < M + 31. Word c*W + p lies in bank
//     p mod 32, distinct across the warp, so every lookup is conflict-free
//     and each lane accumulates its own row: no cross-lane reduction.
//   * dedup (step 5): a replica entry (v, l) carries v's earlier lists (its
//     primary list, then replica lists in ascending id). It is scanned only
//     if none of them is probed; primary entries are always scanned. Each
//     distinct vector of the probed lists is therefore scanned exactly once,
//     with no hashing and no atomics. The paper's parallel hash with per-entry
//     spinlocks (§5) is replaced because a spinning GPU thread can hang.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <atomic>

#include "../fa_internal.h"
#include "rerank_rows.cuh"
#include "warp_topk.cuh"

namespace fa {

constexpr int BIG_THREADS = 1024;  // CTA-top-n variant (256 < n <= 16384)
constexpr int BIG_WARPS = BIG_THREADS / 32;
constexpr int MAX_PROBE = 512;
constexpr int MAX_D = 1024;
constexpr int MAX_TOPN = 16384;

struct ScanArgs {
    // index
    const uint8_t *codes;
    const uint32_t *list_beg;
    const uint64_t *rep_off;
    const uint32_t *rep_v, *rep_mo;
    const uint8_t *rep_t;
    const uint32_t *mem;
    const float *codebooks;
    int32_t d, M, dsub, nlist;  // M: the scan width (table rows per query)
    int32_t ip;                 // the negated inner product instead of the squared L2
    int32_t Mr;                 // subspaces of the index (M rounded up is the scan width)
    int32_t has_rep;
    // batch
    const float *q;
    const int32_t *probes;
    const int32_t *npq;
    const int32_t *ntopq;
    int64_t nq;
    int32_t nprobe, probe_stride, ntop;
    int32_t lut_prec;
    const void *lut;
    const float *lut_scale;
    uint64_t *topkeys;
    int32_t *stats;
    uint32_t *err;
    uint32_t *tile_ctr;
    int32_t persistent;
    const int32_t *order;  // [nq] processing order, or null
    // tiled (batching) form: tiles of at most *tile_T chunks of one query
    const uint32_t *tile_prefix;  // [nq+1] first tile of each query, or null (one CTA per query)
    const uint32_t *tile_T;       // chunks per tile (device scalar)
    uint64_t *partial;            // [tile capacity][ntop] per-tile top-n
    float tau_sigma;              // standard deviations of the CTA top-n threshold estimate
    int32_t sorted_out;           // CTA top-n rows must come out sorted
    const uint32_t *nq_dev;       // device-side query count (slots >= it are done), or null
    uint64_t *selbuf;             // selecting scan: [grid][sel_cap] keys per CTA
    uint32_t sel_cap;
    int32_t *redo;                // selecting scan: queries left to the CTA top-n
    // selecting scan with the exhaustive re-rank fused (rows in internal order)
    int32_t fuse_rr, raw_u8, k, rr_batch;
    const void *raw;
    const int64_t *perm;
    const int32_t *kq;
    int64_t *out_ids;
    float *out_dist;
};

// One unit of scan work: the chunks [c0, climit) of query qi, written to row
// `row` of the output (the query itself, or its tile in the partial buffer).
struct Work {
    int64_t qi, row;
    uint32_t c0, climit;
    int first;  // the query's first tile (writes the gathered count)
};

// Shared memory plan (bytes), shared by host and device. `tail` is the
// per-variant region: per-warp merge buffers, or the CTA key buffer.
// The probed-list set of a query (the replica dedup rule's lookups): a
// bitmap of nlist bits up to 65536 lists (8 KB); beyond that an
// open-addressing table of the probed list ids, 2^pset entries >= 2 nprobe
// (4 KB at nprobe 512 instead of a 32 KB bitmap at 262144 lists).
__host__ __device__ inline int pset_bits(int nlist, int nprobe) {
    if (nlist <= 65536) return 0;
    int b = 4;
    while ((1 << b) < 2 * nprobe) ++b;
    return b;
}

struct ScanSmem {
    int lut, qv, pref, seg, bitmap, tail, total, pset;
    __host__ __device__ ScanSmem(int W, int d, int nlist, int has_rep, int nprobe, int tail_bytes) {
        lut = 256 * W * 4;
        qv = ((d + 3) & ~3) * 4;
        pref = ((2 * nprobe + 1) * 4 + 15) / 16 * 16;
        seg = 2 * nprobe * 4 * 2;
        pset = pset_bits(nlist, nprobe);
        bitmap = !has_rep ? 0 : (pset ? ((4 << pset) + 15) / 16 * 16 : ((nlist + 127) / 128) * 16);
        tail = tail_bytes;
        total = lut + qv + pref + seg + bitmap + tail;
    }
};

struct ScanPtrs {
    float *lut, *qv;
    uint32_t *pref, *seg_beg, *seg_end, *bitmap;  // bitmap: the probed-list set
    unsigned char *tail;
    int pset;  // 0: bitmap; else log2 of the table's entries
    __device__ ScanPtrs(unsigned char *smem, const ScanSmem &p, int nprobe) : pset(p.pset) {
        lut = reinterpret_cast<float *>(smem);
        qv = reinterpret_cast<float *>(smem + p.lut);
        pref = reinterpret_cast<uint32_t *>(smem + p.lut + p.qv);
        seg_beg = reinterpret_cast<uint32_t *>(smem + p.lut + p.qv + p.pref);
        seg_end = seg_beg + 2 * nprobe;
        bitmap = reinterpret_cast<uint32_t *>(smem + p.lut + p.qv + p.pref + p.seg);
        tail = smem + p.lut + p.qv + p.pref + p.seg + p.bitmap;
    }
};

// Builds the LUT of query qi in shared memory (rows of W floats; entry
// p of row c is LUT[p mod M][c] for p < M + 31).
template <int M, int W>
__device__ __forceinline__ void build_lut(const ScanArgs &a, int64_t qi, float *lut, const float *qv) {
    const int dsub = a.dsub;
    constexpr int P = M + 31;
    if (a.lut_prec >= 0) {
        // table from HBM ([M][256] per query): each thread takes 8 consecutive
        // centroids of one subspace with one or two vector loads; the lanes of
        // a warp hold different subspaces, so the shared-memory stores below
        // stay conflict-free
        const int64_t qbase = qi * (int64_t)M * 256;
        for (int idx = threadIdx.x; idx < M * 32; idx += blockDim.x) {
            const int m = idx % M, c0 = (idx / M) * 8;
            const float *sc = a.lut_scale + qi * 2 * M + 2 * m;  // (scale, offset) of subspace m
            const int64_t e0 = qbase + (int64_t)m * 256 + c0;
            float v[8];
            if (a.lut_prec == FA_LUT_F32) {
                const float4 x0 = __ldg(reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(a.lut) + e0));
                const float4 x1 = __ldg(reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(a.lut) + e0) + 1);
                v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
                v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
            } else if (a.lut_prec == FA_LUT_F16) {
                const uint4 u = __ldg(reinterpret_cast<const uint4 *>(reinterpret_cast<const __half *>(a.lut) + e0));
                const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const __half2 h = *reinterpret_cast<const __half2 *>(&w4[j]);
                    v[2 * j] = __half2float(__low2half(h)) * sc[0] + sc[1];
                    v[2 * j + 1] = __half2float(__high2half(h)) * sc[0] + sc[1];
                }
            } else {
                const uint2 u = __ldg(reinterpret_cast<const uint2 *>(reinterpret_cast<const uint8_t *>(a.lut) + e0));
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    __nv_fp8_e4m3 f;
                    f.__x = (uint8_t)(((j < 4 ? u.x : u.y) >> (8 * (j & 3))) & 0xffu);
                    v[j] = float(f) * sc[0] + sc[1];
                }
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int p = 0; p < P; p += M)
                    if (p + m < P) lut[(c0 + j) * W + p + m] = v[j];
        }
        return;
    }
    for (int idx = threadIdx.x; idx < 256 * M; idx += blockDim.x) {
        const int c = idx / M, m = idx - c * M;  // M is a compile-time constant
        // FP32 form: the table built here from the codebooks (Eq. 1); the
        // padding subspaces (m >= Mr) add 0
        float val = 0.f;
        if (m < a.Mr) {
            const float *cw = a.codebooks + ((int64_t)m * 256 + c) * dsub;
            const float *qm = qv + m * dsub;
            for (int j = 0; j < dsub; ++j) {
                if (a.ip) {
                    val = fmaf(-qm[j], cw[j], val);
                } else {
                    const float t = qm[j] - cw[j];
                    val = fmaf(t, t, val);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < P; p += M)
            if (p + m < P) lut[c * W + p + m] = val;
    }
}

template <int M>
__device__ __forceinline__ void load_codes(const uint8_t *codes, uint32_t v, bool valid,
                                           uint32_t (&w)[M / 4]) {
    const uint8_t *row = codes + (size_t)v * M;
    if (valid) {
        if (M % 32 == 0) {
            // one 256-bit load per 32 bytes: a warp reads 32 consecutive rows as
            // one contiguous span (half the L1 wavefronts of 16-byte loads)
#pragma unroll
            for (int i = 0; i < M / 32; ++i) {
                const uint32_t *p = reinterpret_cast<const uint32_t *>(row) + 8 * i;
                asm("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                    : "=r"(w[8 * i + 0]), "=r"(w[8 * i + 1]), "=r"(w[8 * i + 2]),
                      "=r"(w[8 * i + 3]), "=r"(w[8 * i + 4]), "=r"(w[8 * i + 5]),
                      "=r"(w[8 * i + 6]), "=r"(w[8 * i + 7])
                    : "l"(p));
            }
        } else if (M % 16 == 0) {
            const uint4 *p = reinterpret_cast<const uint4 *>(row);
#pragma unroll
            for (int i = 0; i < M / 16; ++i) {
                const uint4 x = __ldg(p + i);
                w[4 * i + 0] = x.x;
                w[4 * i + 1] = x.y;
                w[4 * i + 2] = x.z;
                w[4 * i + 3] = x.w;
            }
        } else {
            const uint2 *p = reinterpret_cast<const uint2 *>(row);
#pragma unroll
            for (int i = 0; i < M / 8; ++i) {
                const uint2 x = __ldg(p + i);
                w[2 * i + 0] = x.x;
                w[2 * i + 1] = x.y;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < M / 4; ++i) w[i] = 0;
    }
}

// ADC distance (Eq. 1) of one rotated code row (rotation r = v mod 32): step
// t sums into accumulator t mod 4 (M is even), and the four are added as
// (a0 + a1) + (a2 + a3). Scalar FP32 adds: the packed two-lane add measured
// more instructions per lookup (its operand pairs) and a slower scan.
template <int M, int W>
__device__ __forceinline__ float adc_words(const uint32_t (&w)[M / 4], uint32_t v, const float *lut) {
    static_assert(M % 2 == 0, "M must be even");
    const uint32_t r4 = (v & 31u) * 4u;
    const char *lb = reinterpret_cast<const char *>(lut);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int t = 0; t < M; ++t) {
        uint32_t off;
        if (W == 64) {
            // (code << 8) | r4 in one byte permute: byte0 <- r4, byte1 <- code
            off = __byte_perm(w[t >> 2], r4, 0x5504u | ((uint32_t)(t & 3) << 4));
        } else {
            const uint32_t c = __byte_perm(w[t >> 2], 0u, 0x4440u | (uint32_t)(t & 3));
            off = c * (uint32_t)(W * 4) + r4;
        }
        acc[t & 3] += *reinterpret_cast<const float *>(lb + off + 4 * t);
    }
    return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// Segment walk state of one warp: the bounds of its current segment, kept in
// registers and refreshed only when a chunk crosses into a later segment.
struct SegCursor {
    int sg = -1;
    uint32_t p0 = 0, p1 = 0, beg = 0, end = 0;
};

// Whether list l is in the query's probed-list set.
__device__ __forceinline__ bool pset_has(const ScanPtrs &S, uint32_t l) {
    if (S.pset == 0) return (S.bitmap[l >> 5] >> (l & 31)) & 1u;
    const uint32_t mask = (1u << S.pset) - 1u;
    uint32_t h = (l * 2654435761u) >> (32 - S.pset);
    for (uint32_t i = 0; i <= mask; ++i) {
        const uint32_t e = S.bitmap[h];
        if (e == l + 1u) return true;
        if (e == 0u) return false;
        h = (h + 1u) & mask;
    }
    return false;
}

// Candidate of this lane in chunk g (32 consecutive entries of one segment):
// primary segments give internal ids directly; replica entries apply the dedup
// rule. Chunks of a warp are visited in increasing order, so the cursor only
// moves forward.
__device__ __forceinline__ void locate(const ScanArgs &a, const ScanPtrs &S, int np, uint32_t g,
                                       SegCursor &c, uint32_t &v, bool &valid) {
    const int lane = threadIdx.x & 31;
    if (c.sg < 0 || g >= c.p1) {
        int sg = c.sg;
        if (sg < 0) {  // first chunk: the last segment that starts at or before g
            int lo = 0, hi = 2 * np - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (S.pref[mid] <= g) lo = mid;
                else hi = mid - 1;
            }
            sg = lo;
        }
        while (g >= S.pref[sg + 1]) ++sg;
        c.sg = sg;
        c.p0 = S.pref[sg];
        c.p1 = S.pref[sg + 1];
        c.beg = S.seg_beg[sg];
        c.end = S.seg_end[sg];
    }
    const uint32_t pos = c.beg + ((g - c.p0) << 5) + lane;
    valid = pos < c.end;
    v = pos;
    if (c.sg >= np && valid) {
        v = a.rep_v[pos];
        const uint32_t mo = a.rep_mo[pos];
        const int t = a.rep_t[pos];
        for (int u = 0; u < t; ++u) {
            const uint32_t l = a.mem[mo + u];
            if (pset_has(S, l)) valid = false;
        }
    }
}

// Per-query set-up shared by both variants: query, segment bounds, probed-list
// bitmap, chunk prefix over 2*np segments, LUT. Ends with a CTA barrier.
template <int M, int W>
__device__ __forceinline__ void query_setup(const ScanArgs &a, const ScanPtrs &S, int64_t qi,
                                            int np) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t *pr = a.probes + qi * a.probe_stride;
    for (int j = threadIdx.x; j < a.d; j += blockDim.x) S.qv[j] = a.q[qi * a.d + j];
    if (a.has_rep) {
        const int words = S.pset ? (1 << S.pset) : (a.nlist + 31) / 32;
        for (int j = threadIdx.x; j < words; j += blockDim.x) S.bitmap[j] = 0u;
    }
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const int l = pr[i];
        if (l < 0 || l >= a.nlist) {
            atomicOr(a.err, DEV_ERR_BOUNDS);
            S.seg_beg[i] = S.seg_end[i] = 0;
            S.seg_beg[np + i] = S.seg_end[np + i] = 0;
            continue;
        }
        S.seg_beg[i] = a.list_beg[l];
        S.seg_end[i] = a.list_beg[l + 1];
        if (a.has_rep) {
            S.seg_beg[np + i] = (uint32_t)a.rep_off[l];
            S.seg_end[np + i] = (uint32_t)a.rep_off[l + 1];
        } else {
            S.seg_beg[np + i] = S.seg_end[np + i] = 0;
        }
    }
    __syncthreads();
    if (a.has_rep)
        for (int i = threadIdx.x; i < np; i += blockDim.x) {
            const int l = pr[i];
            if (l < 0 || l >= a.nlist) continue;
            if (S.pset == 0) {
                atomicOr(&S.bitmap[l >> 5], 1u << (l & 31));
                continue;
            }
            // table insert (the set holds at most half its entries)
            const uint32_t mask = (1u << S.pset) - 1u;
            uint32_t h = ((uint32_t)l * 2654435761u) >> (32 - S.pset);
            for (uint32_t t = 0; t <= mask; ++t) {
                const uint32_t old = atomicCAS(&S.bitmap[h], 0u, (uint32_t)l + 1u);
                if (old == 0u || old == (uint32_t)l + 1u) break;
                h = (h + 1u) & mask;
            }
        }
    if (warp == 0) {
        const int nseg = 2 * np;
        const int per = (nseg + 31) / 32;
        uint32_t loc = 0;
        for (int t = 0; t < per; ++t) {
            const int s = lane * per + t;
            if (s < nseg) loc += (S.seg_end[s] - S.seg_beg[s] + 31u) >> 5;
        }
        uint32_t inc = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        uint32_t run = inc - loc;
        for (int t = 0; t < per; ++t) {
            const int s = lane * per + t;
            if (s < nseg) {
                S.pref[s] = run;
                run += (S.seg_end[s] - S.seg_beg[s] + 31u) >> 5;
            }
        }
        if (lane == 31) S.pref[nseg] = inc;
    }
    build_lut<M, W>(a, qi, S.lut, S.qv);
    __syncthreads();
}

__device__ __forceinline__ void write_stats(const ScanArgs &a, const ScanPtrs &S, int64_t qi,
                                            int np, uint32_t kept) {
    int64_t gathered = 0;
    for (int s = 0; s < 2 * np; ++s) gathered += S.seg_end[s] - S.seg_beg[s];
    a.stats[qi * 4 + 0] = (int32_t)gathered;
    a.stats[qi * 4 + 1] = (int32_t)kept;
}

// Next work slot of this CTA; slot i scans query order[i] (queries grouped by
// their nearest list so that CTAs running together share probed lists in L2).
__device__ __forceinline__ int64_t next_query(const ScanArgs &a, int64_t it) {
    const int64_t slot =
        a.persistent ? (int64_t)atomicAdd(a.tile_ctr, 1u) : (int64_t)blockIdx.x + it * gridDim.x;
    if (slot >= a.nq || (a.nq_dev && slot >= (int64_t)*a.nq_dev)) return a.nq;
    return a.order ? (int64_t)a.order[slot] : slot;
}

// Next unit of work (thread 0 only). Tiled form: slot t is tile t; its query
// is found by binary search in the per-query tile prefix.
__device__ __forceinline__ Work next_work(const ScanArgs &a, int64_t it) {
    Work w;
    if (!a.tile_prefix) {
        w.qi = next_query(a, it);
        w.row = w.qi;
        w.c0 = 0;
        w.climit = 0xffffffffu;
        w.first = 1;
        return w;
    }
    const int64_t slot =
        a.persistent ? (int64_t)atomicAdd(a.tile_ctr, 1u) : (int64_t)blockIdx.x + it * gridDim.x;
    const uint32_t ntiles = a.tile_prefix[a.nq];
    if (slot >= ntiles) {
        w.qi = a.nq;
        return w;
    }
    int64_t lo = 0, hi = a.nq - 1;  // largest q with prefix[q] <= slot
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (a.tile_prefix[mid] <= (uint32_t)slot) lo = mid;
        else hi = mid - 1;
    }
    const uint32_t T = *a.tile_T;
    const uint32_t j = (uint32_t)slot - a.tile_prefix[lo];
    w.qi = lo;
    w.row = slot;
    w.c0 = j * T;
    w.climit = w.c0 + T;
    w.first = j == 0;
    return w;
}

// ---------------------------------------------------------------------------
// Variant 1: n <= 256. Each warp keeps its own top-n in registers; the warps
// share the best n-th key seen by any of them as a common filter threshold.
// A warp works on ILP chunks at a time and loads the code rows of its next
// ILP chunks while scanning the current ones. NT (threads per CTA) and ILP
// are picked per index by the autotuner.
// ---------------------------------------------------------------------------
template <int M, int W, int R, int NT, int ILP>
__global__ void __launch_bounds__(NT, NT == 256 ? 3 : 2) k_scan(const ScanArgs a) {
    constexpr int NWARP = NT / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    const ScanSmem plan(W, a.d, a.nlist, a.has_rep, a.nprobe, NWARP * 64 * 8);
    const ScanPtrs S(smem, plan, a.nprobe);
    uint64_t *wbuf = reinterpret_cast<uint64_t *>(S.tail);
    __shared__ Work s_w;
    __shared__ uint32_t s_kept;
    __shared__ unsigned long long s_thr;
    __shared__ unsigned long long s_slots[NWARP];  // each warp's ceil(n / NWARP)-th key
    constexpr int NW = M / 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int64_t it = 0;; ++it) {
        if (threadIdx.x == 0) {
            s_w = next_work(a, it);
            s_kept = 0;
            s_thr = KEY_INF;
        }
        if (threadIdx.x < NWARP) s_slots[threadIdx.x] = KEY_INF;
        __syncthreads();
        const Work wk = s_w;
        const int64_t qi = wk.qi;
        if (qi >= a.nq) break;
        int np = a.npq ? a.npq[qi] : a.nprobe;
        np = np < 1 ? 1 : (np > a.nprobe ? a.nprobe : np);
        const int ntop = a.ntopq ? a.ntopq[qi] : a.ntop;
        query_setup<M, W>(a, S, qi, np);

        WarpTopK<R> tk;
        tk.init(wbuf + warp * 64, ntop);
        tk.sthr = &s_thr;
        tk.slots = s_slots;
        tk.nslots = NWARP;
        tk.slot = warp;
        const uint32_t total = S.pref[2 * np];
        const uint32_t cend = total < wk.climit ? total : wk.climit;
        uint32_t kept = 0;
        SegCursor sg;
        uint32_t vc[ILP];
        bool okc[ILP];
        uint32_t wc[ILP][NW];
#pragma unroll
        for (int j = 0; j < ILP; ++j) {
            const uint32_t gj = wk.c0 + warp + j * NWARP;
            vc[j] = 0;
            okc[j] = false;
            if (gj < cend) locate(a, S, np, gj, sg, vc[j], okc[j]);
            load_codes<M>(a.codes, vc[j], okc[j], wc[j]);
        }
        for (uint32_t g = wk.c0 + warp; g < cend; g += ILP * NWARP) {
            uint32_t vn[ILP];
            bool okn[ILP];
            uint32_t wn[ILP][NW];
#pragma unroll
            for (int j = 0; j < ILP; ++j) {
                const uint32_t gn = g + (ILP + j) * NWARP;
                vn[j] = 0;
                okn[j] = false;
                if (gn < cend) locate(a, S, np, gn, sg, vn[j], okn[j]);
                load_codes<M>(a.codes, vn[j], okn[j], wn[j]);
            }
            float dist[ILP];
#pragma unroll
            for (int j = 0; j < ILP; ++j) dist[j] = adc_words<M, W>(wc[j], vc[j], S.lut);
#pragma unroll
            for (int j = 0; j < ILP; ++j) {
                kept += okc[j] ? 1u : 0u;
                tk.push(make_key(dist[j], vc[j]), okc[j]);
                vc[j] = vn[j];
                okc[j] = okn[j];
#pragma unroll
                for (int i = 0; i < NW; ++i) wc[j][i] = wn[j][i];
            }
        }
        tk.finish();
        if (a.stats) {
            for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(FULL, kept, o);
            if (lane == 0) atomicAdd(&s_kept, kept);
        }
        __syncthreads();  // LUT no longer needed: reuse it for the merge
        uint64_t *mrg = reinterpret_cast<uint64_t *>(smem);
#pragma unroll
        for (int r = 0; r < R; ++r) mrg[warp * 32 * R + r * 32 + lane] = tk.L[r];
        __syncthreads();
        if (warp == 0) {
            uint64_t L[R];
#pragma unroll
            for (int r = 0; r < R; ++r) L[r] = mrg[r * 32 + lane];
            for (int w = 1; w < NWARP; ++w) {
                uint64_t B[R];
#pragma unroll
                for (int r = 0; r < R; ++r) B[r] = mrg[w * 32 * R + r * 32 + lane];
                merge_sorted<R>(L, B);
            }
            uint64_t *out = (a.tile_prefix ? a.partial : a.topkeys) + wk.row * (int64_t)a.ntop;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int e = r * 32 + lane;
                if (e < a.ntop) out[e] = e < ntop ? L[r] : KEY_INF;
            }
            if (a.stats && lane == 0) {
                if (!a.tile_prefix) {
                    write_stats(a, S, qi, np, s_kept);
                } else {
                    atomicAdd(&a.stats[qi * 4 + 1], (int32_t)s_kept);
                    if (wk.first) {
                        int64_t gathered = 0;
                        for (int sgi = 0; sgi < 2 * np; ++sgi) gathered += S.seg_end[sgi] - S.seg_beg[sgi];
                        a.stats[qi * 4 + 0] = (int32_t)gathered;
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Variant 2: 256 < n <= 16384. The CTA keeps region A = its current top-n
// (sorted, NP = next power of two >= n keys) and region B = new keys below the
// threshold (the n-th key of A), NB <= NP keys (a power of two; NB < NP only
// when two full regions do not fit in shared memory beside the LUT).
//   * Fill phase: the first keys go straight into A; when A may overflow in
//     the next round (or the query ends), A is padded with +inf and sorted
//     once, which sets the threshold.
//   * Then, when B may overflow in the next round, B is sorted and merged
//     into A: with B padded by +inf to NP keys, min(A[i], B[NP-1-i]) is
//     bitonic and holds the NP smallest of both, and only its last NB
//     positions can differ from A; a bitonic merge sorts it.
//   * Threshold estimate: when the query has many more candidates than n, a
//     strided sample of its chunks is scored first and a high quantile of the
//     sample (about n/total of it plus four standard deviations) becomes an
//     initial filter tau. Only keys at or below tau enter A and B, so far
//     fewer keys are sorted and merged. If fewer than n keys fall below tau,
//     the query is scanned again without it, so the result is exact either
//     way.
// Warps scan in lock-step rounds so that every thread reaches the same
// barriers; each warp loads its next round's code rows before it scores the
// current ones, so the loads are in flight across the barriers.
// ---------------------------------------------------------------------------
// In-register bitonic stages of level `size` on the 64-key block starting at
// e0 (lane holds keys e0 + lane and e0 + 32 + lane), strides `from` (<= 32)
// down to 1; key e is sorted ascending where (e & size) == 0.
__device__ __forceinline__ void block64_stages(uint64_t &v0, uint64_t &v1, int e0, int size,
                                               int from) {
    const int lane = threadIdx.x & 31;
    if (from >= 32) {  // partners e and e + 32 sit in one lane
        const bool up = ((e0 + lane) & size) == 0;
        const uint64_t lo = umin64(v0, v1), hi = umax64(v0, v1);
        v0 = up ? lo : hi;
        v1 = up ? hi : lo;
        from = 16;
    }
    const bool up0 = ((e0 + lane) & size) == 0, up1 = ((e0 + 32 + lane) & size) == 0;
    for (int t = from; t >= 1; t >>= 1) {
        const bool lower = (lane & t) == 0;
        const uint64_t o0 = shfl_xor64(v0, t), o1 = shfl_xor64(v1, t);
        v0 = (lower == up0) ? umin64(v0, o0) : umax64(v0, o0);
        v1 = (lower == up1) ? umin64(v1, o1) : umax64(v1, o1);
    }
}

// One shared-memory bitonic stage (stride >= 64) of level `size` over n keys.
__device__ __forceinline__ void smem_stage(uint64_t *x, int n, int size, int stride) {
    for (int i = threadIdx.x; i < n / 2; i += blockDim.x) {
        const int lo = ((i & ~(stride - 1)) << 1) | (i & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const uint64_t p = x[lo], q = x[hi];
        if ((p > q) == up) {
            x[lo] = q;
            x[hi] = p;
        }
    }
    __syncthreads();
}

// Strides 32..1 of level `size` (>= 64) on every 64-key block, in registers.
__device__ __forceinline__ void smem_block_tail(uint64_t *x, int n, int size) {
    const int lane = threadIdx.x & 31;
    for (int b = threadIdx.x >> 5; b < n / 64; b += blockDim.x >> 5) {
        uint64_t v0 = x[b * 64 + lane], v1 = x[b * 64 + 32 + lane];
        block64_stages(v0, v1, b * 64, size, 32);
        x[b * 64 + lane] = v0;
        x[b * 64 + 32 + lane] = v1;
    }
    __syncthreads();
}

// Sorts n keys ascending (n a power of two, >= 64). Levels up to 64 keys and
// the strides below 64 of every later level run in registers, one warp per
// 64-key block; only the longer strides go through shared memory.
__device__ __forceinline__ void smem_bitonic_sort(uint64_t *x, int n) {
    const int lane = threadIdx.x & 31;
    for (int b = threadIdx.x >> 5; b < n / 64; b += blockDim.x >> 5) {
        uint64_t v0 = x[b * 64 + lane], v1 = x[b * 64 + 32 + lane];
        for (int size = 2; size <= 64; size <<= 1) block64_stages(v0, v1, b * 64, size, size >> 1);
        x[b * 64 + lane] = v0;
        x[b * 64 + 32 + lane] = v1;
    }
    __syncthreads();
    for (int size = 128; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride >= 64; stride >>= 1) smem_stage(x, n, size, stride);
        smem_block_tail(x, n, size);
    }
}

// Sorts a bitonic sequence of n keys ascending (n a power of two, >= 64).
__device__ __forceinline__ void smem_bitonic_merge(uint64_t *x, int n) {
    for (int stride = n >> 1; stride >= 64; stride >>= 1) smem_stage(x, n, n, stride);
    smem_block_tail(x, n, n);  // every key index is below n: all ascending
}

// Merges the first cntB keys of B (NB long) into A (NP long, NB <= NP);
// updates the threshold (never above tau).
__device__ __forceinline__ void cta_merge(uint64_t *A, uint64_t *B, int NP, int NB, uint32_t cntB,
                                          int ntop, uint64_t tau, unsigned long long *s_thr,
                                          uint32_t *s_cnt) {
    for (int i = cntB + threadIdx.x; i < NB; i += blockDim.x) B[i] = KEY_INF;
    __syncthreads();
    smem_bitonic_sort(B, NB);
    for (int j = threadIdx.x; j < NB; j += blockDim.x) {
        const uint64_t b = B[j];
        if (b < A[NP - 1 - j]) A[NP - 1 - j] = b;
    }
    __syncthreads();
    smem_bitonic_merge(A, NP);
    if (threadIdx.x == 0) {
        *s_thr = umin64(A[ntop - 1], tau);
        *s_cnt = 0;
    }
    __syncthreads();
}

// Pads A[c, NP) with +inf, sorts it and takes the threshold from it: the end
// of the fill phase, in which new keys go straight into A.
__device__ __forceinline__ void cta_seal(uint64_t *A, int NP, uint32_t c, int ntop, uint64_t tau,
                                         unsigned long long *s_thr, uint32_t *s_cnt,
                                         uint32_t *s_fill) {
    for (int i = c + threadIdx.x; i < NP; i += blockDim.x) A[i] = KEY_INF;
    __syncthreads();
    smem_bitonic_sort(A, NP);
    if (threadIdx.x == 0) {
        *s_thr = umin64(A[ntop - 1], tau);
        *s_cnt = 0;
        *s_fill = 0;
    }
    __syncthreads();
}

// Bits of k at and above bit b (b <= 64).
__device__ __forceinline__ uint64_t high_bits(uint64_t k, int b) { return b >= 64 ? 0ull : k >> b; }

// The r-th smallest (1-based, 1 <= r <= n1 + n2) of the keys x1[0, n1) and
// x2[0, n2) in shared memory, by radix selection: digits of up to 11 bits from the highest bit
// in which the smallest and largest keys differ, each pass counting the keys
// that share the digits chosen so far (hist: 2048 counters). It stops as soon
// as the chosen digits single out one key. Every thread returns the key.
__device__ uint64_t cta_select_rth(const uint64_t *x1, int n1, const uint64_t *x2, int n2, int r,
                                   uint32_t *hist,
                                   unsigned long long *s_lo, unsigned long long *s_hi,
                                   uint32_t *s_dig, uint32_t *s_want, uint32_t *s_cnt) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        *s_lo = ~0ull;
        *s_hi = 0ull;
    }
    __syncthreads();
    uint64_t lo = ~0ull, hi = 0ull;
    for (int i = threadIdx.x; i < n1 + n2; i += blockDim.x) {
        const uint64_t k = i < n1 ? x1[i] : x2[i - n1];
        lo = umin64(lo, k);
        hi = umax64(hi, k);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = umin64(lo, shfl_xor64(lo, o));
        hi = umax64(hi, shfl_xor64(hi, o));
    }
    if (lane == 0) {
        atomicMin(s_lo, (unsigned long long)lo);
        atomicMax(s_hi, (unsigned long long)hi);
    }
    __syncthreads();
    lo = *s_lo;
    hi = *s_hi;
    __syncthreads();
    if (lo == hi) return lo;
    int bound = 64 - __clzll((long long)(lo ^ hi));  // bits >= bound are shared by all keys
    uint64_t prefix = high_bits(lo, bound);
    uint32_t want = (uint32_t)r;
    for (;;) {
        const int width = bound < 11 ? bound : 11, shift = bound - width;
        const uint32_t nb = 1u << width;
        for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < n1 + n2; i += blockDim.x) {
            const uint64_t k = i < n1 ? x1[i] : x2[i - n1];
            if (high_bits(k, bound) == prefix) atomicAdd(&hist[(uint32_t)(k >> shift) & (nb - 1)], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            // lane j sums bins [j * per, (j + 1) * per); the lane whose range
            // holds the want-th key walks its bins
            const uint32_t per = (nb + 31) / 32;
            uint32_t sum = 0;
            for (uint32_t b = lane * per; b < (lane + 1) * per && b < nb; ++b) sum += hist[b];
            uint32_t inc = sum;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(FULL, inc, o);
                if (lane >= o) inc += t;
            }
            const uint32_t before = inc - sum;
            if (before < want && want <= inc) {
                uint32_t run = before;
                for (uint32_t b = lane * per; b < (lane + 1) * per && b < nb; ++b) {
                    if (run + hist[b] >= want) {
                        *s_dig = b;
                        *s_want = want - run;
                        *s_cnt = hist[b];
                        break;
                    }
                    run += hist[b];
                }
            }
        }
        __syncthreads();
        prefix = (prefix << width) | *s_dig;
        want = *s_want;
        const uint32_t cnt = *s_cnt;
        bound = shift;
        __syncthreads();
        if (bound == 0) return prefix;
        if (cnt == 1) {  // the one key with these high bits
            for (int i = threadIdx.x; i < n1 + n2; i += blockDim.x) {
                const uint64_t k = i < n1 ? x1[i] : x2[i - n1];
                if (high_bits(k, bound) == prefix) *s_lo = k;
            }
            __syncthreads();
            const uint64_t k = *s_lo;
            __syncthreads();
            return k;
        }
    }
}

// Upper-bound estimate tau of the query's ntop-th smallest distance, from a
// strided sample of `sch` chunks (keys in buf, sch * 32 of them): the m-th
// smallest sampled distance, m = e + sigma sqrt(e) + 1 (sigma = 4 unless a
// test sets it) for the e = ntop * sch / total sampled keys expected below
// the true ntop-th (found by radix selection). It is only a filter:
// the CTA checks afterwards that ntop keys fell below it and otherwise scans
// the query again without it. Returns the key (tau, max id), or +inf.
template <int M, int W>
__device__ __forceinline__ uint64_t sample_tau(const ScanArgs &a, const ScanPtrs &S, int np,
                                               uint32_t total, int ntop, int sch, uint64_t *buf,
                                               uint32_t *hist, unsigned long long *s_tau,
                                               uint32_t *sel) {
    constexpr int NW = M / 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t stride = total / (uint32_t)sch;
    const int nw = blockDim.x >> 5;
    SegCursor sc;
    // two chunks per warp at a time, both loaded before either is scored
    for (int j = warp; j < sch; j += 2 * nw) {
        const int j2 = j + nw;
        uint32_t v, v2 = 0;
        bool ok, ok2 = false;
        locate(a, S, np, (uint32_t)j * stride, sc, v, ok);
        if (j2 < sch) locate(a, S, np, (uint32_t)j2 * stride, sc, v2, ok2);
        uint32_t w[NW], w2[NW];
        load_codes<M>(a.codes, v, ok, w);
        load_codes<M>(a.codes, v2, ok2, w2);
        const float dist = adc_words<M, W>(w, v, S.lut);
        buf[j * 32 + lane] = ok ? ((uint64_t)f2o(dist) << 32) : KEY_INF;
        if (j2 < sch) {
            const float dist2 = adc_words<M, W>(w2, v2, S.lut);
            buf[j2 * 32 + lane] = ok2 ? ((uint64_t)f2o(dist2) << 32) : KEY_INF;
        }
    }
    __syncthreads();
    const double e = (double)ntop * (double)sch / (double)total;
    const double me = ceil(e + (double)a.tau_sigma * sqrt(e) + 1.0);
    const int m = me < 1.0 ? 1 : (me > 1e9 ? 1000000000 : (int)me);
    if (m > sch * 32) return KEY_INF;
    const uint64_t t =
        cta_select_rth(buf, sch * 32, nullptr, 0, m, hist, s_tau, s_tau + 1, sel, sel + 1, sel + 2);
    return t == KEY_INF ? KEY_INF : (t | 0xffffffffull);
}

template <int M, int W>
__global__ void __launch_bounds__(BIG_THREADS) k_scan_cta(const ScanArgs a, int NP, int NB) {
    extern __shared__ __align__(16) unsigned char smem[];
    const ScanSmem plan(W, a.d, a.nlist, a.has_rep, a.nprobe, (NP + NB) * 8);
    const ScanPtrs S(smem, plan, a.nprobe);
    uint64_t *A = reinterpret_cast<uint64_t *>(S.tail);
    uint64_t *B = A + NP;
    __shared__ int64_t s_q;
    __shared__ uint32_t s_kept, s_cnt, s_fill, s_ovf, s_sel[3];
    __shared__ unsigned long long s_thr, s_sel64[2];
    constexpr int NW = M / 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t round = BIG_WARPS * 32;  // keys one round can add
    // sample chunks for the threshold estimate (the sample lives in A and B;
    // its key count, sch * 32, is a power of two for the sort)
    int sch_max = 256;
    while (sch_max * 32 + 1024 > NP + NB) sch_max >>= 1;  // 1024 keys' room for the histogram

    for (int64_t it = 0;; ++it) {
        if (threadIdx.x == 0) s_q = next_query(a, it);
        __syncthreads();
        const int64_t qi = s_q;
        if (qi >= a.nq) break;
        int np = a.npq ? a.npq[qi] : a.nprobe;
        np = np < 1 ? 1 : (np > a.nprobe ? a.nprobe : np);
        int ntop = a.ntopq ? a.ntopq[qi] : a.ntop;
        ntop = ntop < 1 ? 1 : (ntop > NP ? NP : ntop);
        query_setup<M, W>(a, S, qi, np);

        const uint32_t total = S.pref[2 * np];
        // a threshold estimate pays off only when most candidates are rejected
        uint64_t tau = KEY_INF;
        int sch = sch_max;
        while (sch > 64 && (uint32_t)(2 * sch) > total) sch >>= 1;
        if (total >= 2u * (uint32_t)sch && (uint64_t)total * 32 >= 3ull * (uint64_t)ntop)
            tau = sample_tau<M, W>(a, S, np, total, ntop, sch, A,
                                   reinterpret_cast<uint32_t *>(A + sch * 32), s_sel64, s_sel);

        uint32_t kept = 0;
        // free: warps scan without barriers and append every key at or below
        // tau (about n of them) to A and then B, which are sorted and merged
        // once at the end. Lock-step: the rounds above, with the threshold
        // tightening as A fills. The lock-step scan runs without tau when
        // fewer than n keys fell below it, and with tau when more than A and
        // B hold did.
        bool free_scan = tau != KEY_INF;
        bool written = false;  // the row went out unsorted, straight from the selection
        for (int pass = 0; pass < 3; ++pass) {
            if (threadIdx.x == 0) {
                s_kept = 0;
                s_cnt = 0;
                s_fill = 1;
                s_ovf = 0;
                s_thr = tau;
            }
            __syncthreads();
            kept = 0;
            SegCursor sg;
            // the code rows of this warp's chunk are loaded one chunk ahead
            uint32_t v = 0, w[NW];
            bool ok = false;
            if ((uint32_t)warp < total) locate(a, S, np, warp, sg, v, ok);
            load_codes<M>(a.codes, v, ok && (uint32_t)warp < total, w);
            if (free_scan) {
                // keys beyond A and B spill to the query's output row and, once
                // the scan is done, to the table's shared memory (less 8 KB for
                // the selection's histogram)
                const uint32_t cap = (uint32_t)(NP + NB);
                const uint32_t lut_keys = (uint32_t)(plan.lut / 8) - 1024u;
                uint32_t spill = lut_keys < (uint32_t)a.ntop ? lut_keys : (uint32_t)a.ntop;
                spill = spill < (uint32_t)NP ? spill : (uint32_t)NP;  // merged as a region of <= NP
                uint64_t *row = a.topkeys + qi * (int64_t)a.ntop;
                // scores one chunk's keys and appends those at or below tau
                auto score = [&](const uint32_t (&wc)[NW], uint32_t vc, bool okc) {
                    const float dist = adc_words<M, W>(wc, vc, S.lut);
                    kept += okc ? 1u : 0u;
                    const uint64_t key = make_key(dist, vc);
                    const bool pass_ = okc && key < tau;
                    const uint32_t m = __ballot_sync(FULL, pass_);
                    if (m) {
                        uint32_t p0 = 0;
                        if (lane == 0) p0 = atomicAdd(&s_cnt, (uint32_t)__popc(m));
                        p0 = __shfl_sync(FULL, p0, 0);
                        const uint32_t at = p0 + __popc(m & ((1u << lane) - 1u));
                        if (pass_) {
                            if (at < cap) A[at] = key;  // A and B are contiguous
                            else if (at < cap + spill) row[at - cap] = key;
                            else s_ovf = 1;
                        }
                    }
                };
                // two code buffers in turn: each chunk's rows load while the
                // previous chunk is scored
                for (uint32_t g = warp; g < total; g += 2 * BIG_WARPS) {
                    const uint32_t g1 = g + BIG_WARPS, g2 = g1 + BIG_WARPS;
                    uint32_t v1 = 0, w1[NW];
                    bool ok1 = false;
                    if (g1 < total) locate(a, S, np, g1, sg, v1, ok1);
                    load_codes<M>(a.codes, v1, ok1 && g1 < total, w1);
                    score(w, v, ok);
                    if (g1 >= total) break;
                    ok = false;
                    v = 0;
                    if (g2 < total) locate(a, S, np, g2, sg, v, ok);
                    load_codes<M>(a.codes, v, ok && g2 < total, w);
                    score(w1, v1, ok1);
                }
                __syncthreads();
                const uint32_t c = s_cnt;
                if (s_ovf) {
                    free_scan = false;  // more keys below tau than shared memory holds
                    __syncthreads();
                    continue;
                }
                // the spilled keys move into the table's shared memory
                const uint32_t c1 = c < cap ? c : cap, c2 = c - c1;
                uint64_t *X2 = reinterpret_cast<uint64_t *>(S.lut);
                for (uint32_t i = threadIdx.x; i < c2; i += blockDim.x) X2[i] = row[i];
                __syncthreads();
                if (!a.sorted_out && c >= (uint32_t)ntop) {
                    // the ntop smallest of the c keys, in any order: select the
                    // ntop-th and keep every key up to it
                    const uint64_t kth =
                        cta_select_rth(A, (int)c1, X2, (int)c2, ntop, reinterpret_cast<uint32_t *>(X2 + spill),
                                       s_sel64, s_sel64 + 1, s_sel, s_sel + 1, s_sel + 2);
                    if (threadIdx.x == 0) s_cnt = 0;
                    __syncthreads();
                    for (uint32_t i0 = 0; i0 < c; i0 += blockDim.x) {
                        const uint32_t i = i0 + threadIdx.x;
                        const uint64_t k = i < c1 ? A[i] : (i < c ? X2[i - c1] : KEY_INF);
                        const bool keep = i < c && k <= kth;
                        const uint32_t m = __ballot_sync(FULL, keep);
                        if (m) {
                            uint32_t p0 = 0;
                            if (lane == 0) p0 = atomicAdd(&s_cnt, (uint32_t)__popc(m));
                            p0 = __shfl_sync(FULL, p0, 0);
                            if (keep) row[p0 + __popc(m & ((1u << lane) - 1u))] = k;
                        }
                    }
                    for (int e = ntop + threadIdx.x; e < a.ntop; e += blockDim.x) row[e] = KEY_INF;
                    written = true;
                    __syncthreads();
                    break;
                }
                cta_seal(A, NP, c1 < (uint32_t)NP ? c1 : (uint32_t)NP, ntop, tau, &s_thr, &s_cnt, &s_fill);
                if (c1 > (uint32_t)NP) cta_merge(A, B, NP, NB, c1 - NP, ntop, tau, &s_thr, &s_cnt);
                if (c2 > 0) {
                    int N2 = 64;
                    while ((uint32_t)N2 < c2) N2 <<= 1;  // <= spill < the table's keys
                    cta_merge(A, X2, NP, N2, c2, ntop, tau, &s_thr, &s_cnt);
                }
            } else {
                for (uint32_t base = 0; base < total; base += BIG_WARPS) {
                    const uint32_t g = base + warp, gn = g + BIG_WARPS;
                    uint32_t vn = 0, wn[NW];
                    bool okn = false;
                    if (gn < total) locate(a, S, np, gn, sg, vn, okn);
                    load_codes<M>(a.codes, vn, okn && gn < total, wn);
                    if (g < total) {
                        const float dist = adc_words<M, W>(w, v, S.lut);
                        kept += ok ? 1u : 0u;
                        const uint64_t key = make_key(dist, v);
                        const bool pass_ = ok && key < *(volatile unsigned long long *)&s_thr;
                        const uint32_t m = __ballot_sync(FULL, pass_);
                        if (m) {
                            uint32_t p0 = 0;
                            if (lane == 0) p0 = atomicAdd(&s_cnt, (uint32_t)__popc(m));
                            p0 = __shfl_sync(FULL, p0, 0);
                            // fill phase: straight into A; afterwards into B
                            uint64_t *dst = *(volatile uint32_t *)&s_fill ? A : B;
                            if (pass_) dst[p0 + __popc(m & ((1u << lane) - 1u))] = key;
                        }
                    }
                    v = vn;
                    ok = okn;
#pragma unroll
                    for (int i = 0; i < NW; ++i) w[i] = wn[i];
                    __syncthreads();
                    const uint32_t c = s_cnt, fill = s_fill;
                    __syncthreads();  // every thread has read c before the next round adds to it
                    if (fill) {
                        if (c + round > (uint32_t)NP) cta_seal(A, NP, c, ntop, tau, &s_thr, &s_cnt, &s_fill);
                    } else if (c + round > (uint32_t)NB) {
                        cta_merge(A, B, NP, NB, c, ntop, tau, &s_thr, &s_cnt);
                    }
                }
                __syncthreads();
                const uint32_t c = s_cnt;
                if (s_fill) cta_seal(A, NP, c, ntop, tau, &s_thr, &s_cnt, &s_fill);
                else if (c > 0) cta_merge(A, B, NP, NB, c, ntop, tau, &s_thr, &s_cnt);
            }
            // A holds only keys at or below tau: the top-ntop is exact iff
            // ntop of them were found; otherwise scan again without tau
            if (tau == KEY_INF || A[ntop - 1] != KEY_INF) break;
            tau = KEY_INF;
            free_scan = false;
            __syncthreads();
        }
        if (a.stats) {
            for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(FULL, kept, o);
            if (lane == 0) atomicAdd(&s_kept, kept);
        }
        if (!written) {
            uint64_t *out = a.topkeys + qi * (int64_t)a.ntop;
            for (int e = threadIdx.x; e < a.ntop; e += blockDim.x) out[e] = e < ntop ? A[e] : KEY_INF;
        }
        __syncthreads();
        if (a.stats && threadIdx.x == 0) write_stats(a, S, qi, np, s_kept);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Variant 3 (selecting scan): 256 < n <= 16384 with rows that may come out
// unsorted. Two 512-thread CTAs per SM, so that one CTA's per-query set-up,
// sampling and selection overlap the other's scan. Per query: the sampled
// threshold estimate tau (as in variant 2), a barrier-free scan that appends
// every key at or below tau to this CTA's region of selbuf in global memory
// (L2-resident; about 1.1 n keys, room for 2 n), a radix selection of the
// n-th key over that region and a compaction of the n keys up to it into the
// output row; a query with no more candidates than the region holds keeps
// them all, without an estimate. A query it cannot finish this way (no
// useful sample, fewer than n keys below tau, or more than the region holds)
// is appended to the redo list, which variant 2 then scans.
// ---------------------------------------------------------------------------
constexpr int SEL_THREADS = 512;
constexpr int SEL_WARPS = SEL_THREADS / 32;

// Algorithm 1 with eps < 0 (no early stop) on the query's kept candidates
// (the keys of buf[0, c) up to kth, kept_n of them), fused into the scan:
// the result is the exact top-k by (squared L2, caller id) of all of them,
// so the order they are taken in does not matter. Each warp re-ranks every
// 16th group of 32 into its own sorted top-32 (raw rows in HBM in internal
// order; the caller id is looked up only for keys that can enter it), then
// warp 0 merges the 16 lists and writes the caller ids and distances. Ends
// with a CTA barrier. uint8 rows of a multiple of 16 bytes only.
__device__ __forceinline__ void rerank_fused(const ScanArgs &a, const ScanPtrs &S, int64_t qi,
                                          const uint64_t *buf, uint32_t c, uint64_t kth, int kept_n,
                                          uint32_t *scratch, uint32_t *s_small) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t *wq = reinterpret_cast<uint64_t *>(scratch);            // [SEL_WARPS][32]
    uint32_t *qp = reinterpret_cast<uint32_t *>(wq + SEL_WARPS * 32);  // [d / 4]
    if (warp == 0) {
        bool qint = false;
        if (!a.ip && a.d <= 258 && a.d % 16 == 0) qint = pack_u8_query(S.qv, a.d, qp);
        if (lane == 0) s_small[1] = qint ? 1u : 0u;
    }
    __syncthreads();
    const bool qint = s_small[1] != 0;
    int kk = a.kq ? a.kq[qi] : a.k;
    kk = kk < 1 ? 1 : (kk > a.k ? a.k : kk);
    uint64_t Q[1] = {KEY_INF};
    const uint8_t *raw = static_cast<const uint8_t *>(a.raw);
    // each lane's row of the warp's next group of 32 keys is prefetched into
    // L2 while this group's rows are read and scored: the rows are scattered,
    // so a group otherwise waits a full DRAM round trip (two groups ahead
    // measured no better)
    auto prefetch_row = [&](uint32_t j) {
        if (j < c) {
            const uint64_t kj = buf[j];
            if (kj <= kth) {
                const uint8_t *r = raw + (int64_t)(uint32_t)(kj & 0xffffffffu) * a.d;
                for (int o = 0; o < a.d; o += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(r + o));
            }
        }
    };
    prefetch_row((uint32_t)warp * 32 + lane);
    for (uint32_t i0 = (uint32_t)warp * 32; i0 < c; i0 += SEL_THREADS) {
        const uint32_t i = i0 + lane;
        const uint64_t key = i < c ? buf[i] : KEY_INF;
        const int64_t v = (i < c && key <= kth) ? (int64_t)(uint32_t)(key & 0xffffffffu) : (int64_t)-1;
        prefetch_row(i + SEL_THREADS);
        const float dist = qint ? (a.d % 32 == 0 ? exact_rows_u8int32(raw, a.d, qp, v)
                                                 : exact_rows_u8int<uint4>(raw, a.d, qp, v))
                                : (a.ip ? exact_rows<uint8_t, uint4, true>(raw, a.d, S.qv, v)
                                        : exact_rows<uint8_t, uint4>(raw, a.d, S.qv, v));
        const uint64_t kthq = shfl64(Q[0], kk - 1);
        const bool maybe = v >= 0 && f2o(dist) <= (uint32_t)(kthq >> 32);
        uint64_t nk[1] = {maybe ? make_key(dist, (uint32_t)a.perm[v]) : KEY_INF};
        const uint32_t in = __ballot_sync(FULL, nk[0] < kthq);
        if (__popc(in) > 8) {  // many new keys (the first groups): sort and merge
            bitonic_sort<1>(nk);
            merge_sorted32<1>(Q, nk[0]);
        } else if (in) {
            insert_sorted32(Q[0], nk[0], in);
        }
    }
    wq[warp * 32 + lane] = Q[0];
    __syncthreads();
    if (warp == 0) {
        uint64_t L[1] = {wq[lane]};
        for (int w2 = 1; w2 < SEL_WARPS; ++w2) merge_sorted32<1>(L, wq[w2 * 32 + lane]);
        if (lane < a.k) {
            const uint64_t key = lane < kk ? L[0] : KEY_INF;
            a.out_ids[qi * a.k + lane] = key == KEY_INF ? -1 : (int64_t)(key & 0xffffffffu);
            a.out_dist[qi * a.k + lane] = key == KEY_INF ? INFINITY : o2f((uint32_t)(key >> 32));
        }
        if (a.stats && lane == 0) {
            a.stats[qi * 4 + 2] = (kept_n + a.rr_batch - 1) / a.rr_batch;
            a.stats[qi * 4 + 3] = kept_n;
        }
    }
    __syncthreads();
}

template <int M, int W>
__global__ void __launch_bounds__(SEL_THREADS, 2) k_scan_sel(const ScanArgs a, int sch_max) {
    extern __shared__ __align__(16) unsigned char smem[];
    const ScanSmem plan(W, a.d, a.nlist, a.has_rep, a.nprobe, sch_max * 32 * 8 + 8192);
    const ScanPtrs S(smem, plan, a.nprobe);
    uint64_t *samp = reinterpret_cast<uint64_t *>(S.tail);
    uint32_t *hist = reinterpret_cast<uint32_t *>(samp + sch_max * 32);
    uint64_t *buf = a.selbuf + (int64_t)blockIdx.x * a.sel_cap;
    __shared__ int64_t s_q;
    __shared__ uint32_t s_cnt, s_kept, s_sel[3];
    __shared__ unsigned long long s_sel64[2];
    constexpr int NW = M / 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int64_t it = 0;; ++it) {
        if (threadIdx.x == 0) {
            s_q = next_query(a, it);
            s_cnt = 0;
            s_kept = 0;
        }
        __syncthreads();
        const int64_t qi = s_q;
        if (qi >= a.nq) break;
        int np = a.npq ? a.npq[qi] : a.nprobe;
        np = np < 1 ? 1 : (np > a.nprobe ? a.nprobe : np);
        int ntop = a.ntopq ? a.ntopq[qi] : a.ntop;
        ntop = ntop < 1 ? 1 : (ntop > a.ntop ? a.ntop : ntop);
        query_setup<M, W>(a, S, qi, np);  // ends with a barrier
        const uint32_t total = S.pref[2 * np];
        int sch = sch_max;
        while (sch > 64 && (uint32_t)(2 * sch) > total) sch >>= 1;
        // every candidate fits the buffer: keep them all, no estimate needed
        const bool all = (uint64_t)total * 32 <= (uint64_t)a.sel_cap;
        uint64_t tau = KEY_INF;
        if (!all && total >= 2u * (uint32_t)sch)
            tau = sample_tau<M, W>(a, S, np, total, ntop, sch, samp, hist, s_sel64, s_sel);
        if (!all && tau == KEY_INF) {  // no useful estimate: variant 2 takes the query
            if (threadIdx.x == 0) a.redo[atomicAdd(a.tile_ctr + 3, 1u)] = (int32_t)qi;
            __syncthreads();
            continue;
        }
        uint32_t kept = 0;
        SegCursor sg;
        // warp w scans a consecutive run of the primary chunks, then one of
        // the replica chunks (an equal share of each: replica entries cost
        // more, their dedup lookups), so that its segment cursor moves on
        // only at the end of a list
        const uint32_t nprim = S.pref[np], nrep = total - nprim;
        const uint32_t perp = (nprim + SEL_WARPS - 1) / SEL_WARPS, perr = (nrep + SEL_WARPS - 1) / SEL_WARPS;
        const uint32_t g0 = min(nprim, (uint32_t)warp * perp), gend = min(nprim, g0 + perp);
        const uint32_t r0 = nprim + min(nrep, (uint32_t)warp * perr), rend = min(total, r0 + perr);
        uint32_t v = 0, w[NW];
        bool ok = false;
        if (g0 < gend) locate(a, S, np, g0, sg, v, ok);
        load_codes<M>(a.codes, v, ok && g0 < gend, w);
        // tau = (its distance, the largest id): a key is below it iff its
        // distance is at or below tau's (internal ids stay below 2^32 - 1)
        const uint32_t tau_hi = (uint32_t)(tau >> 32);
        // keys below tau gather in the warp's 64-key stage in shared memory
        // (the sample's room, free until the next query) and go to the CTA
        // buffer 32 at a time: one slot reservation and one coalesced store
        // per 32 keys instead of per chunk
        uint64_t *stage = samp + warp * 64;
        uint32_t scnt = 0;  // keys in the stage (warp-uniform, < 32 between chunks)
        const uint32_t lt = (1u << lane) - 1u;
        auto flush = [&](uint32_t n) {
            __syncwarp();
            uint32_t p0 = 0;
            if (lane == 0) p0 = atomicAdd(&s_cnt, n);
            p0 = __shfl_sync(FULL, p0, 0);
            if ((uint32_t)lane < n && p0 + lane < a.sel_cap) buf[p0 + lane] = stage[lane];
        };
        auto score = [&](const uint32_t (&wc)[NW], uint32_t vc, bool okc) {
            const float dist = adc_words<M, W>(wc, vc, S.lut);
            const uint32_t dk = f2o(dist);
            const bool pass_ = okc && dk <= tau_hi;
            const uint32_t m = __ballot_sync(FULL, pass_);
            if (m) {
                if (pass_) stage[scnt + __popc(m & lt)] = ((uint64_t)dk << 32) | vc;
                scnt += (uint32_t)__popc(m);
                if (scnt >= 32) {
                    flush(32);
                    const uint64_t rest = stage[lane + 32];  // the scnt - 32 keys after them
                    __syncwarp();
                    scnt -= 32;
                    if ((uint32_t)lane < scnt) stage[lane] = rest;
                }
            }
        };
        for (uint32_t g = g0; g < gend; g += 2) {
            const uint32_t g1 = g + 1, g2 = g + 2;
            uint32_t v1 = 0, w1[NW];
            bool ok1 = false;
            if (g1 < gend) locate(a, S, np, g1, sg, v1, ok1);
            load_codes<M>(a.codes, v1, ok1 && g1 < gend, w1);
            score(w, v, ok);
            if (g1 >= gend) break;
            ok = false;
            v = 0;
            if (g2 < gend) locate(a, S, np, g2, sg, v, ok);
            load_codes<M>(a.codes, v, ok && g2 < gend, w);
            score(w1, v1, ok1);
        }
        // every primary entry is kept; replica entries are counted as scanned
        for (uint32_t g = r0; g < rend; ++g) {  // the replica share, one chunk at a time
            ok = false;
            locate(a, S, np, g, sg, v, ok);
            load_codes<M>(a.codes, v, ok, w);
            kept += ok ? 1u : 0u;
            score(w, v, ok);
        }
        if (scnt) flush(scnt);
        if (a.stats) {
            for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(FULL, kept, o);
            if (threadIdx.x == 0)
                for (int sgi = 0; sgi < np; ++sgi) kept += S.seg_end[sgi] - S.seg_beg[sgi];
            if (lane == 0) atomicAdd(&s_kept, kept);
        }
        __syncthreads();
        const uint32_t c = s_cnt;
        if ((!all && c < (uint32_t)ntop) || c > a.sel_cap) {  // tau too low or too high
            if (threadIdx.x == 0) a.redo[atomicAdd(a.tile_ctr + 3, 1u)] = (int32_t)qi;
            __syncthreads();
            continue;
        }
        // the ntop-th key, or every key when the query has no more than ntop
        const uint64_t kth = c > (uint32_t)ntop
                                 ? cta_select_rth(buf, (int)c, nullptr, 0, ntop, hist, s_sel64, s_sel64 + 1,
                                                  s_sel, s_sel + 1, s_sel + 2)
                                 : KEY_INF;
        const int kept_n = c < (uint32_t)ntop ? (int)c : ntop;
        if (a.fuse_rr) {
            if (a.stats && threadIdx.x == 0) write_stats(a, S, qi, np, s_kept);
            rerank_fused(a, S, qi, buf, c, kth, kept_n, hist, s_sel);
            continue;
        }
        uint64_t *row = a.topkeys + qi * (int64_t)a.ntop;
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        for (uint32_t i0 = 0; i0 < c; i0 += blockDim.x) {
            const uint32_t i = i0 + threadIdx.x;
            const uint64_t k = i < c ? buf[i] : KEY_INF;
            const bool keep = i < c && k <= kth;
            const uint32_t m = __ballot_sync(FULL, keep);
            if (m) {
                uint32_t p0 = 0;
                if (lane == 0) p0 = atomicAdd(&s_cnt, (uint32_t)__popc(m));
                p0 = __shfl_sync(FULL, p0, 0);
                if (keep) row[p0 + __popc(m & ((1u << lane) - 1u))] = k;
            }
        }
        for (int e = kept_n + threadIdx.x; e < a.ntop; e += blockDim.x) row[e] = KEY_INF;
        __syncthreads();
        if (a.stats && threadIdx.x == 0) write_stats(a, S, qi, np, s_kept);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Batched form: the whole batch scanned list by list (steps 3-7 for many
// queries at once). Each (query, probed list) pair of the batch goes in its
// list's bucket; a unit of work is one list (or a tile of T chunks of a long
// list) with two of the queries that probe it. The unit's CTA builds a
// shared-memory table whose 32-bit words hold both queries' FP16 entries, in
// the rotated layout of the scans above, reads each code row of the list once
// and takes both queries' distances from one lookup per code byte, adding the
// FP16 entries in FP32. The entries share one scale per query (s_q) beside a
// per-subspace offset o_q[m], so that
//   ADC(q, v) = s_q * sum_m e_q[m][code_m(v)] + sum_m o_q[m].
// Every key at or below the query's sampled threshold is appended to the
// query's buffer in global memory; a per-query kernel then selects the top-n
// by radix selection and, for an exhaustive re-rank of uint8 rows in HBM,
// re-ranks them. Queries the threshold does not serve (fewer than n keys or
// more than the buffer below it, or no useful sample) go on the redo list,
// which the per-query scans take.
//
// Dedup (step 5) follows the same probe-set rule: a replica entry (v, l) is
// kept for a query unless one of v's earlier lists is in that query's probe
// bitmap (global memory here, one bit per list).
// ---------------------------------------------------------------------------
constexpr int BQ_THREADS = 384;  // list scan: 12 warps per CTA
constexpr int BQ_GMAX = 4;       // queries per unit: two FP16 or four FP8 entries per table word

struct BatchArgs {
    const uint8_t *codes;
    const uint32_t *list_beg;
    const uint64_t *rep_off;
    const uint32_t *rep_v, *rep_mo;
    const uint8_t *rep_t;
    const uint32_t *mem;
    const uint32_t *lorder;  // [nlist] lists by decreasing chunk count
    int32_t M, nlist, has_rep, nlw;
    // the sub-batch: queries q0 .. q0 + nq - 1 of the call
    const int32_t *probes;  // [call nq][stride]
    const int32_t *npq;
    int64_t q0, nq;
    int32_t nprobe, stride;
    const void *lut;        // [call nq][M][256] FP16 or FP8, one scale per query
    int32_t G;              // queries per unit (entries per table word): 2 FP16, 4 FP8
    const float *qsum;      // [call nq][2]: s_q, sum of the offsets
    const uint64_t *tau;    // [call nq] threshold keys (0: the query is redone)
    uint32_t *lcnt, *lqoff, *lcur;  // [nlist], [nlist + 1], [nlist]
    int32_t *lq;            // queries of each list, bucket by bucket
    uint32_t *upre;         // [nlist + 1] units before each list rank
    uint32_t *pbits;        // [call nq][nlw] probed lists
    uint32_t *cnt;          // [call nq] keys appended
    uint64_t *buf;          // [call nq][cap]
    uint32_t cap, T;
    int32_t *stats;
    uint32_t *err;
    uint32_t *ctr;          // unit counter
};

__device__ __forceinline__ int bq_np(const BatchArgs &b, int64_t q) {
    int np = b.npq ? b.npq[q] : b.nprobe;
    return np < 1 ? 1 : (np > b.nprobe ? b.nprobe : np);
}

// one thread per (query, probe rank): bucket sizes and probe bitmaps
__global__ void k_bq_count(const BatchArgs b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.nq * b.nprobe) return;
    const int64_t q = b.q0 + i / b.nprobe;
    const int j = (int)(i % b.nprobe);
    if (j >= bq_np(b, q)) return;
    const int l = b.probes[q * b.stride + j];
    if (l < 0 || l >= b.nlist) {
        atomicOr(b.err, DEV_ERR_BOUNDS);
        return;
    }
    atomicAdd(&b.lcnt[l], 1u);
    if (b.has_rep) atomicOr(&b.pbits[q * b.nlw + (l >> 5)], 1u << (l & 31));
}

__global__ void k_bq_scatter(const BatchArgs b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.nq * b.nprobe) return;
    const int64_t q = b.q0 + i / b.nprobe;
    const int j = (int)(i % b.nprobe);
    if (j >= bq_np(b, q)) return;
    const int l = b.probes[q * b.stride + j];
    if (l < 0 || l >= b.nlist) return;
    b.lq[atomicAdd(&b.lcur[l], 1u)] = (int32_t)q;
}

__device__ __forceinline__ uint32_t bq_chunks(const BatchArgs &b, int l) {
    uint32_t c = (b.list_beg[l + 1] - b.list_beg[l] + 31u) >> 5;
    if (b.has_rep) c += (uint32_t)((b.rep_off[l + 1] - b.rep_off[l] + 31u) >> 5);
    return c;
}

// Exclusive scan of f(i), i < n, by one CTA: out[i] (and out2[i]) = sum of
// f(j) for j < i, out[n] = the total.
template <class F>
__device__ void cta_excl_scan(int n, F f, uint32_t *out, uint32_t *out2, uint32_t *ws) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int i0 = threadIdx.x * per, i1 = min(n, i0 + per);
    uint32_t loc = 0;
    for (int i = i0; i < i1; ++i) loc += f(i);
    uint32_t inc = loc;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t x = lane < nw ? ws[lane] : 0u;
        uint32_t xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, xi, o);
            if (lane >= o) xi += y;
        }
        ws[lane] = xi - x;
        if (lane == 31) ws[32] = xi;
    }
    __syncthreads();
    uint32_t run = ws[warp] + inc - loc;
    for (int i = i0; i < i1; ++i) {
        out[i] = run;
        if (out2) out2[i] = run;
        run += f(i);
    }
    if (threadIdx.x == 0) out[n] = ws[32];
    __syncthreads();
}

// One CTA: bucket offsets, and units per list rank (query groups x chunk tiles).
__global__ void __launch_bounds__(1024) k_bq_plan(const BatchArgs b) {
    __shared__ uint32_t ws[33];
    cta_excl_scan(b.nlist, [&](int l) { return b.lcnt[l]; }, b.lqoff, b.lcur, ws);
    cta_excl_scan(
        b.nlist,
        [&](int r) {
            const int l = (int)b.lorder[r];
            const uint32_t nql = b.lcnt[l], nch = bq_chunks(b, l);
            if (nql == 0 || nch == 0) return 0u;
            return ((nql + b.G - 1) / b.G) * ((nch + b.T - 1) / b.T);
        },
        b.upre, nullptr, ws);
}

// Appends the keys of one chunk at or below the query's threshold to its buffer.
// The threshold is a full (distance, id) key, so a run of equal distances at
// the threshold is split by id as the sample split it.
__device__ __forceinline__ void bq_append(const BatchArgs &b, int64_t q, float dist, uint32_t v,
                                          bool ok, uint64_t tau, int lane) {
    const uint32_t od = f2o(dist);
    const bool pass = ok && (((uint64_t)od << 32) | v) <= tau;
    const uint32_t msk = __ballot_sync(FULL, pass);
    if (msk) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&b.cnt[q], (uint32_t)__popc(msk));
        base = __shfl_sync(FULL, base, 0);
        const uint32_t pos = base + __popc(msk & ((1u << lane) - 1u));
        if (pass && pos < b.cap) b.buf[q * (int64_t)b.cap + pos] = ((uint64_t)od << 32) | v;
    }
}

// Unit u of the plan: its list, first and last chunk, and its queries.
struct BqUnit {
    int64_t q[BQ_GMAX];
    uint64_t tau[BQ_GMAX];
    float sc[BQ_GMAX], of[BQ_GMAX];
    uint32_t u, l, c0, c1, nprim;
};

__device__ __forceinline__ void bq_decode(const BatchArgs &b, uint32_t u, uint32_t total_units,
                                          BqUnit &x) {
    x.u = u;
    if (u >= total_units) return;
    int lo = 0, hi = b.nlist - 1;  // the last list rank r with upre[r] <= u
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.upre[mid] <= u) lo = mid;
        else hi = mid - 1;
    }
    const int l = (int)b.lorder[lo];
    const uint32_t r = u - b.upre[lo];
    const uint32_t nql = b.lcnt[l];
    const uint32_t ngrp = (nql + b.G - 1) / b.G;
    const uint32_t grp = r % ngrp, tile = r / ngrp;  // groups of one tile run side by side
    const uint32_t nch = bq_chunks(b, l);
    x.l = (uint32_t)l;
    x.nprim = (b.list_beg[l + 1] - b.list_beg[l] + 31u) >> 5;
    x.c0 = tile * b.T;
    x.c1 = min(nch, (tile + 1) * b.T);
    for (int j = 0; j < BQ_GMAX; ++j) {
        const uint32_t k = grp * b.G + j;
        if (j < b.G && k < nql) {
            const int64_t q = b.lq[b.lqoff[l] + k];
            x.q[j] = q;
            x.tau[j] = b.tau[q];
            x.sc[j] = b.qsum[2 * q];
            x.of[j] = b.qsum[2 * q + 1];
        } else {
            x.q[j] = -1;
            x.tau[j] = 0;
            x.sc[j] = 0.f;
            x.of[j] = 0.f;
        }
    }
}

// The E queries' ADC sums of one rotated code row, E entries per table word:
// E = 2, FP16 entries added in FP32; E = 4, FP8 (e4m3) entries converted in
// pairs to half2 and added as half2 over 16 subspaces (at most 16 x 448, well
// inside FP16), then in FP32.
template <int M, int W, int E>
__device__ __forceinline__ void adc_multi(const uint32_t (&w)[M / 4], uint32_t v, const uint32_t *tbl,
                                          float (&acc)[E]) {
    const uint32_t r4 = (v & 31u) * 4u;
    const char *tb = reinterpret_cast<const char *>(tbl);
    if (E == 2) {
        float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
#pragma unroll
        for (int t = 0; t < M; ++t) {
            uint32_t off;
            if (W == 64) {
                off = __byte_perm(w[t >> 2], r4, 0x5504u | ((uint32_t)(t & 3) << 4));
            } else {
                const uint32_t c = __byte_perm(w[t >> 2], 0u, 0x4440u | (uint32_t)(t & 3));
                off = c * (uint32_t)(W * 4) + r4;
            }
            const uint32_t x = *reinterpret_cast<const uint32_t *>(tb + off + 4 * t);
            if (t & 1)
                asm("{.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\tadd.rn.f32.f16 %0, lo, %0;\n\t"
                    "add.rn.f32.f16 %1, hi, %1;}"
                    : "+f"(b0), "+f"(b1)
                    : "r"(x));
            else
                asm("{.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\tadd.rn.f32.f16 %0, lo, %0;\n\t"
                    "add.rn.f32.f16 %1, hi, %1;}"
                    : "+f"(a0), "+f"(a1)
                    : "r"(x));
        }
        acc[0] = a0 + b0;
        acc[1] = a1 + b1;
    } else {
        float f[4] = {0.f, 0.f, 0.f, 0.f};
        uint32_t h01 = 0u, h23 = 0u;  // half2 partial sums of queries (0, 1) and (2, 3)
#pragma unroll
        for (int t = 0; t < M; ++t) {
            uint32_t off;
            if (W == 64) {
                off = __byte_perm(w[t >> 2], r4, 0x5504u | ((uint32_t)(t & 3) << 4));
            } else {
                const uint32_t c = __byte_perm(w[t >> 2], 0u, 0x4440u | (uint32_t)(t & 3));
                off = c * (uint32_t)(W * 4) + r4;
            }
            const uint32_t x = *reinterpret_cast<const uint32_t *>(tb + off + 4 * t);
            asm("{.reg .b16 lo, hi;\n\t.reg .b32 p, r;\n\tmov.b32 {lo, hi}, %2;\n\t"
                "cvt.rn.f16x2.e4m3x2 p, lo;\n\tcvt.rn.f16x2.e4m3x2 r, hi;\n\t"
                "add.rn.f16x2 %0, %0, p;\n\tadd.rn.f16x2 %1, %1, r;}"
                : "+r"(h01), "+r"(h23)
                : "r"(x));
            if ((t & 15) == 15 || t == M - 1) {
                float x0, x1, x2, x3;
                asm("{.reg .b16 a, b, c, d;\n\tmov.b32 {a, b}, %4;\n\tmov.b32 {c, d}, %5;\n\t"
                    "cvt.f32.f16 %0, a;\n\tcvt.f32.f16 %1, b;\n\tcvt.f32.f16 %2, c;\n\tcvt.f32.f16 %3, d;}"
                    : "=f"(x0), "=f"(x1), "=f"(x2), "=f"(x3)
                    : "r"(h01), "r"(h23));
                f[0] += x0;
                f[1] += x1;
                f[2] += x2;
                f[3] += x3;
                h01 = h23 = 0u;
            }
        }
#pragma unroll
        for (int j = 0; j < E; ++j) acc[j] = f[j];
    }
}

// The group table of E queries in shared memory: word (c, p), p < M + 31,
// holds entry [p mod M][c] of each query (query j in byte lane j of the word
// for FP8, half j for FP16; a query slot < 0 holds zeros). A thread takes 16
// centroids of one subspace, so the lanes of a warp store consecutive words.
template <int M, int W, int E>
__device__ __forceinline__ void bq_table(const void *lut, const int64_t (&qs)[E], uint32_t *tbl) {
    constexpr int P = M + 31;
    for (int idx = threadIdx.x; idx < M * 16; idx += blockDim.x) {
        const int m = idx % M, c0 = (idx / M) * 16;
        uint32_t wd[16];
        if (E == 2) {
            uint32_t h[2][8];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
#pragma unroll
                for (int i = 0; i < 8; ++i) h[j][i] = 0u;
                if (qs[j] >= 0) {
                    const uint4 *p = reinterpret_cast<const uint4 *>(
                        static_cast<const __half *>(lut) + (qs[j] * M + m) * 256 + c0);
                    const uint4 x0 = __ldg(p), x1 = __ldg(p + 1);
                    h[j][0] = x0.x; h[j][1] = x0.y; h[j][2] = x0.z; h[j][3] = x0.w;
                    h[j][4] = x1.x; h[j][5] = x1.y; h[j][6] = x1.z; h[j][7] = x1.w;
                }
            }
#pragma unroll
            for (int i = 0; i < 16; ++i)
                wd[i] = __byte_perm(h[0][i >> 1], h[1][i >> 1], (i & 1) ? 0x7632u : 0x5410u);
        } else {
            uint32_t e[4][4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                e[j][0] = e[j][1] = e[j][2] = e[j][3] = 0u;
                if (qs[j] >= 0) {
                    const uint4 x = __ldg(reinterpret_cast<const uint4 *>(
                        static_cast<const uint8_t *>(lut) + (qs[j] * M + m) * 256 + c0));
                    e[j][0] = x.x; e[j][1] = x.y; e[j][2] = x.z; e[j][3] = x.w;
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {  // entries 4i .. 4i + 3 of the four queries
                const uint32_t t0 = __byte_perm(e[0][i], e[1][i], 0x5140u);
                const uint32_t t1 = __byte_perm(e[2][i], e[3][i], 0x5140u);
                const uint32_t t2 = __byte_perm(e[0][i], e[1][i], 0x7362u);
                const uint32_t t3 = __byte_perm(e[2][i], e[3][i], 0x7362u);
                wd[4 * i + 0] = __byte_perm(t0, t1, 0x5410u);
                wd[4 * i + 1] = __byte_perm(t0, t1, 0x7632u);
                wd[4 * i + 2] = __byte_perm(t2, t3, 0x5410u);
                wd[4 * i + 3] = __byte_perm(t2, t3, 0x7632u);
            }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j)
#pragma unroll
            for (int p = 0; p < P; p += M)
                if (p + m < P) tbl[(c0 + j) * W + p + m] = wd[j];
    }
}

// The m-th smallest of a sample of the query's candidate keys, with the
// distances computed exactly as the batched scan computes them (its group
// table with this query alone, adc_multi, then the query's scale and offset
// sum). Each of the sch * 32 sample slots takes one candidate from its own
// chunk, spread evenly over all the query's chunks: the near candidates of a
// query sit in few lists, and whole sampled chunks would leave the estimate
// to the luck of which lists they fell in.
template <int M, int W, int E>
__device__ __forceinline__ uint64_t sample_tau_bq(const ScanArgs &a, const ScanPtrs &S, int np,
                                                  uint32_t total, int ntop, int sch, uint64_t *buf,
                                                  uint32_t *hist, unsigned long long *s_tau,
                                                  uint32_t *sel, const uint32_t *tbl, float scale,
                                                  float offset) {
    constexpr int NW = M / 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t ns = (uint64_t)sch * 32;
    const int nw = blockDim.x >> 5;
    SegCursor sc;  // each lane's chunks increase from one step to the next
    for (int j = warp; j < sch; j += nw) {
        uint32_t v;
        bool ok;
        const uint64_t slot = (uint64_t)j * 32 + lane;
        locate(a, S, np, (uint32_t)(slot * total / ns), sc, v, ok);
        uint32_t w[NW];
        load_codes<M>(a.codes, v, ok, w);
        float acc[E];
        adc_multi<M, W, E>(w, v, tbl, acc);
        buf[j * 32 + lane] = ok ? (((uint64_t)f2o(fmaf(acc[0], scale, offset)) << 32) | v) : KEY_INF;
    }
    __syncthreads();
    // e sampled keys are expected below the query's n-th key. A query handed
    // back costs a whole per-query scan, and for a query of millions of
    // candidates e is well below 1, where sigma * sqrt(e) alone leaves a
    // Poisson tail of ~1e-3; the extra sigma keys bring it below ~1e-8 (for
    // sigma 4) while the keys kept stay a small multiple of n.
    const double e = (double)ntop * (double)sch / (double)total;
    const double me = ceil(e + (double)a.tau_sigma * sqrt(e) + 1.0 + (double)a.tau_sigma);
    const int m = me < 1.0 ? 1 : (me > 1e9 ? 1000000000 : (int)me);
    if (m > sch * 32) return KEY_INF;
    // the m-th full key: keys are distinct, so about m / sample of the scan's
    // keys fall at or below it even where many distances are equal
    return cta_select_rth(buf, sch * 32, nullptr, 0, m, hist, s_tau, s_tau + 1, sel, sel + 1, sel + 2);
}

// Per-query threshold estimate from a strided sample of the query's
// candidates (sample_tau_bq), and the per-query constants the batched scan
// applies: the table's scale s_q and the sum of its offsets. A threshold of 0
// marks a query the list scan cannot serve (no useful sample); +inf keeps
// every candidate.
template <int M, int W, int E>
__global__ void __launch_bounds__(SEL_THREADS, 2) k_bq_tau(const ScanArgs a, uint64_t *tau,
                                                           uint32_t *cnt, float *qsum, uint32_t cap,
                                                           int sch_max) {
    extern __shared__ __align__(16) unsigned char smem[];
    const ScanSmem plan(W, a.d, a.nlist, a.has_rep, a.nprobe, sch_max * 32 * 8 + 8192);
    const ScanPtrs S(smem, plan, a.nprobe);
    uint64_t *samp = reinterpret_cast<uint64_t *>(S.tail);
    uint32_t *hist = reinterpret_cast<uint32_t *>(samp + sch_max * 32);
    __shared__ int64_t s_q;
    __shared__ uint32_t s_sel[3];
    __shared__ unsigned long long s_sel64[2];
    for (int64_t it = 0;; ++it) {
        if (threadIdx.x == 0) s_q = next_query(a, it);
        __syncthreads();
        const int64_t qi = s_q;
        if (qi >= a.nq) break;
        int np = a.npq ? a.npq[qi] : a.nprobe;
        np = np < 1 ? 1 : (np > a.nprobe ? a.nprobe : np);
        int ntop = a.ntopq ? a.ntopq[qi] : a.ntop;
        ntop = ntop < 1 ? 1 : (ntop > a.ntop ? a.ntop : ntop);
        query_setup<M, W>(a, S, qi, np);  // ends with a barrier
        const float *sq = a.lut_scale + qi * 2 * a.M;
        float off = 0.f;
        for (int m = 0; m < a.M; ++m) off += sq[2 * m + 1];
        const uint32_t total = S.pref[2 * np];
        int sch = sch_max;
        while (sch > 64 && (uint32_t)(2 * sch) > total) sch >>= 1;
        const bool all = (uint64_t)total * 32 <= (uint64_t)cap;
        uint64_t t = KEY_INF;
        if (!all) {
            if (total >= 2u * (uint32_t)sch) {
                // this query's group table in place of its FP32 table
                int64_t qs[E];
#pragma unroll
                for (int j = 0; j < E; ++j) qs[j] = j == 0 ? qi : -1;
                uint32_t *tbl = reinterpret_cast<uint32_t *>(S.lut);
                __syncthreads();
                bq_table<M, W, E>(a.lut, qs, tbl);
                __syncthreads();
                t = sample_tau_bq<M, W, E>(a, S, np, total, ntop, sch, samp, hist, s_sel64, s_sel, tbl, sq[0],
                                           off);
            }
            if (t == KEY_INF) t = 0;
        }
        if (threadIdx.x == 0) {
            tau[qi] = t;
            cnt[qi] = 0;
            qsum[2 * qi] = sq[0];
            qsum[2 * qi + 1] = off;
            if (a.stats) {
                int64_t gathered = 0;
                for (int sgi = 0; sgi < 2 * np; ++sgi) gathered += S.seg_end[sgi] - S.seg_beg[sgi];
                a.stats[qi * 4 + 0] = (int32_t)gathered;
                a.stats[qi * 4 + 1] = 0;
            }
        }
        __syncthreads();
    }
}

template <int M, int W, int E>
__global__ void __launch_bounds__(BQ_THREADS) k_bq_scan(const BatchArgs b) {
    extern __shared__ __align__(16) uint32_t tbl[];  // [256][W] words of the E queries' entries
    __shared__ BqUnit s_unit[2];  // the current unit and the next one
    constexpr int NW = M / 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t total_units = b.upre[b.nlist];
    if (threadIdx.x == 0) bq_decode(b, atomicAdd(b.ctr, 1u), total_units, s_unit[0]);
    __syncthreads();
    for (int cur = 0;; cur ^= 1) {
        const BqUnit &U = s_unit[cur];
        if (U.u >= total_units) break;
        const int l = (int)U.l;
        int64_t qs[E];
#pragma unroll
        for (int j = 0; j < E; ++j) qs[j] = U.q[j];
        bq_table<M, W, E>(b.lut, qs, tbl);
        __syncthreads();
        // the next unit is claimed and decoded while this one is scanned
        if (threadIdx.x == 0) bq_decode(b, atomicAdd(b.ctr, 1u), total_units, s_unit[cur ^ 1]);
        uint64_t tq[E];
        float sc[E], of[E];
        uint32_t kept[E];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            tq[j] = U.tau[j];
            sc[j] = U.sc[j];
            of[j] = U.of[j];
            kept[j] = 0u;
        }
        const uint32_t nprim = U.nprim, c1 = U.c1;
        const uint32_t lb0 = b.list_beg[l], lb1 = b.list_beg[l + 1];
        // candidate of this lane in chunk g: primary ids directly, replica
        // entries through the probe-set rule of each query
        auto locate_bq = [&](uint32_t g, uint32_t &v, bool (&ok)[E]) -> bool {
            v = 0;
            bool any = false;
            if (g < nprim) {
                v = lb0 + (g << 5) + lane;
                any = v < lb1;
#pragma unroll
                for (int j = 0; j < E; ++j) ok[j] = any && qs[j] >= 0;
                return any;
            }
            const uint64_t e = b.rep_off[l] + ((uint64_t)(g - nprim) << 5) + lane;
            const bool in = e < b.rep_off[l + 1];
#pragma unroll
            for (int j = 0; j < E; ++j) ok[j] = in && qs[j] >= 0;
            if (in) {
                v = b.rep_v[e];
                const uint32_t mo = b.rep_mo[e];
                const int t = b.rep_t[e];
                for (int u = 0; u < t; ++u) {
                    const uint32_t ll = b.mem[mo + u];
#pragma unroll
                    for (int j = 0; j < E; ++j)
                        if (ok[j] && ((b.pbits[qs[j] * b.nlw + (ll >> 5)] >> (ll & 31)) & 1u)) ok[j] = false;
                }
            }
#pragma unroll
            for (int j = 0; j < E; ++j) any = any || ok[j];
            return any;
        };
        constexpr int NWARP = BQ_THREADS / 32;
        // each warp loads the code rows of its next chunk before it scores the current one
        uint32_t g = U.c0 + warp;
        uint32_t v = 0, w[NW];
        bool ok[E];
        {
            const bool any = g < c1 && locate_bq(g, v, ok);
            if (g >= c1)
#pragma unroll
                for (int j = 0; j < E; ++j) ok[j] = false;
            load_codes<M>(b.codes, v, any, w);
        }
        for (; g < c1; g += NWARP) {
            const uint32_t gn = g + NWARP;
            uint32_t vn = 0, wn[NW];
            bool okn[E];
            const bool anyn = gn < c1 && locate_bq(gn, vn, okn);
            load_codes<M>(b.codes, vn, anyn, wn);
            float acc[E];
            adc_multi<M, W, E>(w, v, tbl, acc);
#pragma unroll
            for (int j = 0; j < E; ++j) {
                kept[j] += ok[j] ? 1u : 0u;
                bq_append(b, qs[j], fmaf(acc[j], sc[j], of[j]), v, ok[j], tq[j], lane);
            }
            v = vn;
#pragma unroll
            for (int i = 0; i < NW; ++i) w[i] = wn[i];
#pragma unroll
            for (int j = 0; j < E; ++j) ok[j] = gn < c1 && okn[j];
        }
        if (b.stats) {
#pragma unroll
            for (int j = 0; j < E; ++j) {
                uint32_t k = kept[j];
                for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(FULL, k, o);
                if (lane == 0 && qs[j] >= 0 && k) atomicAdd(&b.stats[qs[j] * 4 + 1], (int32_t)k);
            }
        }
        __syncthreads();  // the table takes the next unit's queries
    }
}

// Per query: the top-n of its buffer (radix selection of the n-th key), then
// the exhaustive re-rank (fused) or the top-n row (unsorted, or sorted when
// sort_np > 0: an early-stopping re-rank reads it in order). Queries whose
// buffer does not hold their top-n go on the redo list.
__global__ void __launch_bounds__(SEL_THREADS) k_bq_select(const ScanArgs a, const uint64_t *tau,
                                                           const uint32_t *cnt, const uint64_t *bufs,
                                                           uint32_t cap, int sort_np, uint32_t *qctr,
                                                           uint32_t *nredo) {
    extern __shared__ __align__(16) unsigned char smem[];
    const ScanSmem plan(0, a.d, a.nlist, 0, 1, 8192 + sort_np * 8);
    const ScanPtrs S(smem, plan, 1);
    uint32_t *hist = reinterpret_cast<uint32_t *>(S.tail);
    uint64_t *X = reinterpret_cast<uint64_t *>(S.tail + 8192);
    __shared__ int64_t s_q;
    __shared__ uint32_t s_cnt, s_sel[3];
    __shared__ unsigned long long s_sel64[2];
    const int lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t slot = atomicAdd(qctr, 1u);
            s_q = slot < a.nq ? (int64_t)slot : a.nq;
        }
        __syncthreads();
        const int64_t qi = s_q;
        if (qi >= a.nq) break;
        int ntop = a.ntopq ? a.ntopq[qi] : a.ntop;
        ntop = ntop < 1 ? 1 : (ntop > a.ntop ? a.ntop : ntop);
        const uint64_t t = tau[qi];
        const uint32_t c = cnt[qi];
        const bool all = t == KEY_INF;
        if (t == 0 || c > cap || (!all && c < (uint32_t)ntop)) {
            if (threadIdx.x == 0) a.redo[atomicAdd(nredo, 1u)] = (int32_t)qi;
            __syncthreads();
            continue;
        }
        const uint64_t *buf = bufs + qi * (int64_t)cap;
        const uint64_t kth = c > (uint32_t)ntop
                                 ? cta_select_rth(buf, (int)c, nullptr, 0, ntop, hist, s_sel64,
                                                  s_sel64 + 1, s_sel, s_sel + 1, s_sel + 2)
                                 : KEY_INF;
        const int kept_n = c < (uint32_t)ntop ? (int)c : ntop;
        if (a.fuse_rr) {
            for (int j = threadIdx.x; j < a.d; j += blockDim.x) S.qv[j] = a.q[qi * a.d + j];
            __syncthreads();
            rerank_fused(a, S, qi, buf, c, kth, kept_n, hist, s_sel);
            continue;
        }
        uint64_t *row = a.topkeys + qi * (int64_t)a.ntop;
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        for (uint32_t i0 = 0; i0 < c; i0 += blockDim.x) {
            const uint32_t i = i0 + threadIdx.x;
            const uint64_t k = i < c ? buf[i] : KEY_INF;
            const bool keep = i < c && k <= kth;
            const uint32_t m = __ballot_sync(FULL, keep);
            if (m) {
                uint32_t p0 = 0;
                if (lane == 0) p0 = atomicAdd(&s_cnt, (uint32_t)__popc(m));
                p0 = __shfl_sync(FULL, p0, 0);
                const uint32_t at = p0 + __popc(m & ((1u << lane) - 1u));
                if (keep && at < (uint32_t)ntop) {  // keys are distinct: at most ntop pass
                    if (sort_np) X[at] = k;
                    else row[at] = k;
                }
            }
        }
        __syncthreads();
        if (sort_np) {
            for (int e = kept_n + threadIdx.x; e < sort_np; e += blockDim.x) X[e] = KEY_INF;
            __syncthreads();
            smem_bitonic_sort(X, sort_np);
            for (int e = threadIdx.x; e < a.ntop; e += blockDim.x) row[e] = e < kept_n ? X[e] : KEY_INF;
        } else {
            for (int e = kept_n + threadIdx.x; e < a.ntop; e += blockDim.x) row[e] = KEY_INF;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int pow2_at_least(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

template <class K>
static void set_smem(K kfn, int bytes) {
    FA_CHECK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
}

static int scan_grid(const ScanLaunch &l, int smem_total) {
    if (!l.persistent) return (int)(l.nq < (int64_t)INT32_MAX ? l.nq : INT32_MAX);
    int per_sm = (227 * 1024) / (smem_total + 1024);
    per_sm = per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm);
    int grid = cur_num_sms() * per_sm;
    if (l.tile_prefix) return grid;  // tiles outnumber queries
    return (int64_t)grid > l.nq ? (int)l.nq : grid;
}

template <int M, int W, int R, int NT, int ILP>
static void launch_warp_variant(const ScanArgs &a, const ScanLaunch &l, cudaStream_t st) {
    const ScanSmem plan(W, a.d, a.nlist, a.has_rep, a.nprobe, (NT / 32) * 64 * 8);
    FA_REQUIRE((NT / 32) * 32 * R * 8 <= plan.lut, FA_ERR_ARG, "LUT region too small for merge");
    FA_REQUIRE(plan.total <= 227 * 1024, FA_ERR_ARG, "scan shared memory above 227 KB");
    const int grid = scan_grid(l, plan.total);
    set_smem(k_scan<M, W, R, NT, ILP>, plan.total);
    k_scan<M, W, R, NT, ILP><<<grid, NT, plan.total, st>>>(a);
}

template <int M, int W, int R>
static void launch_warp_r(const ScanArgs &a, const ScanLaunch &l, cudaStream_t st) {
    const bool big = l.threads >= 512;
    if (l.ilp >= 2) {
        if (big) launch_warp_variant<M, W, R, 512, 2>(a, l, st);
        else launch_warp_variant<M, W, R, 256, 2>(a, l, st);
    } else {
        if (big) launch_warp_variant<M, W, R, 512, 1>(a, l, st);
        else launch_warp_variant<M, W, R, 256, 1>(a, l, st);
    }
}

template <int M, int W>
static bool launch_scan_m(const ScanArgs &a, const ScanLaunch &l, cudaStream_t st) {
    bool fused = false;
    if (a.ntop <= 256) {
        if (a.ntop <= 32) launch_warp_r<M, W, 1>(a, l, st);
        else if (a.ntop <= 64) launch_warp_r<M, W, 2>(a, l, st);
        else if (a.ntop <= 128) launch_warp_r<M, W, 4>(a, l, st);
        else launch_warp_r<M, W, 8>(a, l, st);
    } else {
        // selecting scan (two CTAs per SM) when the rows may come out unsorted
        // and its buffers are there; variant 2 then takes what it hands back
        // (a 64-chunk sample: 2048 keys; a 128-chunk one measured 1.3 % slower
        // overall, its sampling costing more than its tighter estimate saves)
        constexpr int sch_max = 64;
        static_assert(sch_max * 32 >= SEL_WARPS * 64, "the sample's room holds the warps' key stages");
        const ScanSmem sel_plan(W, a.d, a.nlist, a.has_rep, a.nprobe, sch_max * 32 * 8 + 8192);
        const bool sel = !a.sorted_out && a.selbuf && a.redo && sel_plan.total <= 113 * 1024;
        ScanArgs b = a;  // variant 2's arguments
        if (sel) {
            const int smem_sel = sel_plan.total;
            ScanArgs c = a;
            c.persistent = 1;
            c.sel_cap = 2u * (uint32_t)a.ntop;
            // the exhaustive re-rank rides along when its rows are in HBM in
            // internal order and k fits one warp list
            fused = l.fuse_rerank && a.raw && a.raw_u8 && a.d % 16 == 0 && l.k >= 1 && l.k <= 32 &&
                    l.out_ids && l.out_dist;
            c.fuse_rr = fused ? 1 : 0;
            FA_CHECK_CUDA(cudaMemsetAsync(a.tile_ctr, 0, 4 * sizeof(uint32_t), st));
            set_smem(k_scan_sel<M, W>, smem_sel);
            k_scan_sel<M, W><<<2 * cur_num_sms(), SEL_THREADS, smem_sel, st>>>(c, sch_max);
            FA_CHECK_CUDA(cudaGetLastError());
            // variant 2 over the redo list (its length is on the device)
            b.order = a.redo;
            b.nq_dev = a.tile_ctr + 3;
            b.tile_ctr = a.tile_ctr + 2;
            b.persistent = 1;
        }
        const int NP = pow2_at_least(a.ntop < 2 * BIG_WARPS * 32 ? 2 * BIG_WARPS * 32 : a.ntop);
        // B region: as large as NP while both fit beside the LUT, and at least
        // two rounds of keys
        constexpr int budget = 227 * 1024 - 256;  // room for the kernel's static shared variables
        int NB = NP;
        while (NB > 2 * BIG_WARPS * 32 &&
               ScanSmem(W, a.d, a.nlist, a.has_rep, a.nprobe, (NP + NB) * 8).total > budget)
            NB >>= 1;
        const ScanSmem plan(W, a.d, a.nlist, a.has_rep, a.nprobe, (NP + NB) * 8);
        FA_REQUIRE(plan.total <= budget, FA_ERR_ARG,
                   "scan shared memory above 227 KB (top-n too large for this M)");
        const int grid = sel ? cur_num_sms() : scan_grid(l, plan.total);
        set_smem(k_scan_cta<M, W>, plan.total);
        k_scan_cta<M, W><<<grid, BIG_THREADS, plan.total, st>>>(b, NP, NB);
    }
    FA_CHECK_CUDA(cudaGetLastError());
    return fused;
}

static std::atomic<float> g_tau_sigma{4.0f};

void set_tau_sigma(float sigma) { g_tau_sigma.store(sigma); }

static ScanArgs scan_args(const DeviceIndex &ix, const ScanLaunch &l) {
    FA_REQUIRE(l.nprobe <= MAX_PROBE, FA_ERR_ARG, "nprobe above 512");
    FA_REQUIRE(ix.d <= MAX_D, FA_ERR_ARG, "d above 1024");
    FA_REQUIRE(l.ntop >= 1 && l.ntop <= MAX_TOPN, FA_ERR_ARG, "top-n must be in 1..16384");
    ScanArgs a{};
    a.codes = ix.codes;
    a.list_beg = ix.list_beg;
    a.rep_off = ix.rep_off;
    a.rep_v = ix.rep_v;
    a.rep_mo = ix.rep_mo;
    a.rep_t = ix.rep_t;
    a.mem = ix.mem;
    a.codebooks = ix.codebooks;
    a.d = ix.d;
    a.M = ix.Mp;
    a.Mr = ix.M;
    a.ip = ix.metric == FA_METRIC_IP ? 1 : 0;
    a.dsub = ix.dsub;
    a.nlist = ix.nlist;
    a.has_rep = ix.n_rep > 0 ? 1 : 0;
    a.q = l.q;
    a.probes = l.probes;
    a.npq = l.npq;
    a.ntopq = l.ntopq;
    a.nq = l.nq;
    a.nprobe = l.nprobe;
    a.probe_stride = l.probe_stride;
    a.ntop = l.ntop;
    a.lut_prec = l.lut_prec;
    a.lut = l.lut;
    a.lut_scale = l.lut_scale;
    a.topkeys = l.topkeys;
    a.stats = l.stats;
    a.err = l.err;
    a.tile_ctr = l.tile_ctr;
    a.persistent = l.persistent;
    a.order = l.order;
    a.tile_prefix = l.tile_prefix;
    a.tile_T = l.tile_T;
    a.partial = l.partial;
    a.tau_sigma = g_tau_sigma.load();
    a.sorted_out = l.sorted;
    a.nq_dev = nullptr;
    a.selbuf = l.selbuf;
    a.sel_cap = 0;
    a.redo = l.redo;
    a.fuse_rr = 0;
    a.raw_u8 = ix.raw_dtype == FA_U8 ? 1 : 0;
    a.k = l.k;
    a.rr_batch = l.rerank_batch;
    a.raw = ix.raw_internal ? ix.raw : nullptr;  // fusion reads rows by internal id
    a.perm = ix.perm;
    a.kq = l.kq;
    a.out_ids = l.out_ids;
    a.out_dist = l.out_dist;
    return a;
}

bool launch_scan(const DeviceIndex &ix, const ScanLaunch &l, cudaStream_t st) {
    if (l.nq == 0) return false;
    const ScanArgs a = scan_args(ix, l);
    if (a.tile_prefix) {
        FA_REQUIRE(l.ntop <= 256, FA_ERR_ARG, "the tiled form supports top-n <= 256");
        FA_REQUIRE(l.persistent, FA_ERR_ARG, "the tiled form runs persistent CTAs");
    }
    switch (ix.Mp) {
        case 8: return launch_scan_m<8, 64>(a, l, st);
        case 16: return launch_scan_m<16, 64>(a, l, st);
        case 32: return launch_scan_m<32, 64>(a, l, st);
        case 48: return launch_scan_m<48, 96>(a, l, st);
        case 64: return launch_scan_m<64, 128>(a, l, st);
        default: FA_REQUIRE(false, FA_ERR_ARG, "M must be one of 8, 16, 32, 48, 64");
    }
    return false;
}

// Per-query scans of the queries on the redo list (its length on the
// device): the CTA top-n for n above 256, the per-warp top-n below.
template <int M, int W>
static void launch_redo_m(const ScanArgs &b, cudaStream_t st) {
    ScanLaunch l{};
    l.persistent = 1;
    l.nq = b.nq;
    if (b.ntop <= 256) {
        if (b.ntop <= 32) launch_warp_variant<M, W, 1, 256, 1>(b, l, st);
        else if (b.ntop <= 64) launch_warp_variant<M, W, 2, 256, 1>(b, l, st);
        else if (b.ntop <= 128) launch_warp_variant<M, W, 4, 256, 1>(b, l, st);
        else launch_warp_variant<M, W, 8, 256, 1>(b, l, st);
        return;
    }
    const int NP = pow2_at_least(b.ntop < 2 * BIG_WARPS * 32 ? 2 * BIG_WARPS * 32 : b.ntop);
    constexpr int budget = 227 * 1024 - 256;
    int NB = NP;
    while (NB > 2 * BIG_WARPS * 32 &&
           ScanSmem(W, b.d, b.nlist, b.has_rep, b.nprobe, (NP + NB) * 8).total > budget)
        NB >>= 1;
    const ScanSmem plan(W, b.d, b.nlist, b.has_rep, b.nprobe, (NP + NB) * 8);
    FA_REQUIRE(plan.total <= budget, FA_ERR_ARG,
               "scan shared memory above 227 KB (top-n too large for this M)");
    set_smem(k_scan_cta<M, W>, plan.total);
    k_scan_cta<M, W><<<cur_num_sms(), BIG_THREADS, plan.total, st>>>(b, NP, NB);
    FA_CHECK_CUDA(cudaGetLastError());
}

template <int M, int W>
static bool launch_batched_m(const DeviceIndex &ix, const ScanLaunch &l, const BatchBufs &bb,
                             cudaStream_t st) {
    const ScanArgs a = scan_args(ix, l);
    const int nlw = (ix.nlist + 31) / 32;
    FA_CHECK_CUDA(cudaMemsetAsync(bb.ctr, 0, 8 * sizeof(uint32_t), st));
    FA_CHECK_CUDA(cudaMemsetAsync(l.tile_ctr, 0, 4 * sizeof(uint32_t), st));
    if (a.has_rep) FA_CHECK_CUDA(cudaMemsetAsync(bb.pbits, 0, sizeof(uint32_t) * l.nq * nlw, st));
    // 1. per-query thresholds (a larger sample when the top-n is small)
    {
        const int sch_max = l.ntop <= 256 ? 256 : 64;
        ScanArgs t = a;
        t.persistent = 1;
        t.tile_ctr = bb.ctr;
        t.order = l.order;
        const ScanSmem plan(W, a.d, a.nlist, a.has_rep, a.nprobe, sch_max * 32 * 8 + 8192);
        FA_REQUIRE(plan.total <= 227 * 1024, FA_ERR_ARG, "threshold sample above 227 KB");
        auto ktau = l.lut_prec == FA_LUT_FP8 ? k_bq_tau<M, W, 4> : k_bq_tau<M, W, 2>;
        set_smem(ktau, plan.total);
        ktau<<<2 * cur_num_sms(), SEL_THREADS, plan.total, st>>>(t, bb.tau, bb.cnt, bb.qsum, bb.cap, sch_max);
        FA_CHECK_CUDA(cudaGetLastError());
    }
    // 2. the list scan, sub-batch by sub-batch (the sub-batch's tables stay in L2)
    BatchArgs b{};
    b.codes = ix.codes;
    b.list_beg = ix.list_beg;
    b.rep_off = ix.rep_off;
    b.rep_v = ix.rep_v;
    b.rep_mo = ix.rep_mo;
    b.rep_t = ix.rep_t;
    b.mem = ix.mem;
    b.lorder = ix.lorder;
    b.M = ix.Mp;
    b.nlist = ix.nlist;
    b.has_rep = a.has_rep;
    b.nlw = nlw;
    b.probes = l.probes;
    b.npq = l.npq;
    b.nprobe = l.nprobe;
    b.stride = l.probe_stride;
    b.lut = l.lut;
    b.G = l.lut_prec == FA_LUT_FP8 ? 4 : 2;
    b.qsum = bb.qsum;
    b.tau = bb.tau;
    b.lcnt = bb.lcnt;
    b.lqoff = bb.lqoff;
    b.lcur = bb.lcur;
    b.lq = bb.lq;
    b.upre = bb.upre;
    b.pbits = bb.pbits;
    b.cnt = bb.cnt;
    b.buf = bb.buf;
    b.cap = bb.cap;
    b.T = bb.tile_chunks;
    b.stats = l.stats;
    b.err = l.err;
    b.ctr = bb.ctr + 1;
    const int tsmem = 256 * W * 4;
    auto kscan = b.G == 4 ? k_bq_scan<M, W, 4> : k_bq_scan<M, W, 2>;
    set_smem(kscan, tsmem);
    int per_sm = 0;
    FA_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kscan, BQ_THREADS, tsmem));
    FA_REQUIRE(per_sm >= 1, FA_ERR_ARG, "the batched scan's table does not fit shared memory");
    const int gscan = per_sm * cur_num_sms();
    for (int64_t q0 = 0; q0 < l.nq; q0 += bb.qsub) {
        b.q0 = q0;
        b.nq = std::min<int64_t>(bb.qsub, l.nq - q0);
        FA_CHECK_CUDA(cudaMemsetAsync(bb.lcnt, 0, sizeof(uint32_t) * ix.nlist, st));
        FA_CHECK_CUDA(cudaMemsetAsync(bb.ctr + 1, 0, sizeof(uint32_t), st));
        const int64_t pairs = b.nq * b.nprobe;
        const unsigned g = (unsigned)((pairs + 255) / 256);
        k_bq_count<<<g, 256, 0, st>>>(b);
        k_bq_plan<<<1, 1024, 0, st>>>(b);
        k_bq_scatter<<<g, 256, 0, st>>>(b);
        kscan<<<gscan, BQ_THREADS, tsmem, st>>>(b);
        FA_CHECK_CUDA(cudaGetLastError());
    }
    // 3. selection of each query's top-n, and the exhaustive re-rank fused
    ScanArgs c = a;
    const bool fused = l.fuse_rerank && a.raw && a.raw_u8 && a.d % 16 == 0 && l.k >= 1 && l.k <= 32 &&
                       l.out_ids && l.out_dist;
    c.fuse_rr = fused ? 1 : 0;
    const int sort_np = (!fused && l.sorted) ? pow2_at_least(std::max(64, l.ntop)) : 0;
    const int ssmem = ScanSmem(0, a.d, a.nlist, 0, 1, 8192 + sort_np * 8).total;
    FA_REQUIRE(ssmem <= 227 * 1024, FA_ERR_ARG, "selection shared memory above 227 KB");
    set_smem(k_bq_select, ssmem);
    int sel_sm = 0;
    FA_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sel_sm, k_bq_select, SEL_THREADS, ssmem));
    k_bq_select<<<std::max(1, sel_sm) * cur_num_sms(), SEL_THREADS, ssmem, st>>>(
        c, bb.tau, bb.cnt, bb.buf, bb.cap, sort_np, bb.ctr + 2, l.tile_ctr + 3);
    FA_CHECK_CUDA(cudaGetLastError());
    // 4. the queries handed back, scanned one CTA per query
    ScanArgs r = a;
    r.order = l.redo;
    r.nq_dev = l.tile_ctr + 3;
    r.tile_ctr = l.tile_ctr + 2;
    r.persistent = 1;
    r.fuse_rr = 0;
    launch_redo_m<M, W>(r, st);
    return fused;
}

bool launch_batched(const DeviceIndex &ix, const ScanLaunch &l, const BatchBufs &bb, cudaStream_t st) {
    if (l.nq == 0) return false;
    FA_REQUIRE((l.lut_prec == FA_LUT_F16 || l.lut_prec == FA_LUT_FP8) && l.lut, FA_ERR_ARG,
               "the batched form reads the FP16 or FP8 table");
    FA_REQUIRE(l.redo && l.tile_ctr, FA_ERR_ARG, "the batched form needs its redo list");
    switch (ix.Mp) {
        case 8: return launch_batched_m<8, 64>(ix, l, bb, st);
        case 16: return launch_batched_m<16, 64>(ix, l, bb, st);
        case 32: return launch_batched_m<32, 64>(ix, l, bb, st);
        case 48: return launch_batched_m<48, 96>(ix, l, bb, st);
        case 64: return launch_batched_m<64, 128>(ix, l, bb, st);
        default: FA_REQUIRE(false, FA_ERR_ARG, "M must be one of 8, 16, 32, 48, 64");
    }
    return false;
}

// ---------------------------------------------------------------------------
// Tiled (batching) form, planned on the device so the whole search can be
// captured in a CUDA graph:
//   k_tile_count  chunks of 32 candidates per query (and their total)
//   k_tile_plan   one CTA: chunks per tile T = max(requested, total / room) so
//                 the tiles fit the partial buffer, then the per-query tile
//                 prefix (exclusive scan)
//   k_tile_merge  one warp per query merges its tiles' sorted top-n lists
// ---------------------------------------------------------------------------
__global__ void k_tile_count(const int32_t *probes, const int32_t *npq, int64_t nq, int32_t nprobe,
                             int32_t stride, const uint32_t *list_beg, const uint64_t *rep_off,
                             int32_t nlist, int32_t has_rep, uint32_t *chunks,
                             unsigned long long *total) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (q >= nq) return;
    int np = npq ? npq[q] : nprobe;
    np = np < 1 ? 1 : (np > nprobe ? nprobe : np);
    uint32_t c = 0;
    for (int i = lane; i < np; i += 32) {
        const int l = probes[q * stride + i];
        if (l < 0 || l >= nlist) continue;
        c += (list_beg[l + 1] - list_beg[l] + 31u) >> 5;
        if (has_rep) c += (uint32_t)((rep_off[l + 1] - rep_off[l] + 31u) >> 5);
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if (lane == 0) {
        chunks[q] = c;
        atomicAdd(total, (unsigned long long)c);
    }
}

__global__ void k_tile_plan(const uint32_t *chunks, int64_t nq, uint32_t T_req, uint32_t cap,
                            const unsigned long long *total, uint32_t *T_out, uint32_t *prefix) {
    __shared__ uint32_t part[32];
    __shared__ uint32_t carry;
    __shared__ uint32_t sT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        const unsigned long long room = cap > nq ? (unsigned long long)(cap - nq) : 1ull;
        unsigned long long T = (*total + room - 1) / room;
        if (T < T_req) T = T_req;
        sT = (uint32_t)(T > 0xffffffull ? 0xffffffull : (T < 1 ? 1 : T));
        *T_out = sT;
        carry = 0;
    }
    __syncthreads();
    const uint32_t T = sT;
    for (int64_t base = 0; base < nq; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        uint32_t v = 0;
        if (i < nq) {
            const uint32_t c = chunks[i];
            v = c == 0 ? 1u : (c + T - 1) / T;
        }
        uint32_t inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) part[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            uint32_t pp = lane < (int)(blockDim.x >> 5) ? part[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, pp, o);
                if (lane >= o) pp += y;
            }
            part[lane] = pp;
        }
        __syncthreads();
        const uint32_t excl = carry + (warp ? part[warp - 1] : 0u) + inc - v;
        if (i < nq) prefix[i] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) prefix[nq] = carry;
}

template <int R>
__global__ void __launch_bounds__(256) k_tile_merge(const uint64_t *partial, const uint32_t *prefix,
                                                     int64_t nq, int32_t ntop, uint64_t *topkeys) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * 8 + warp;
    if (q >= nq) return;
    uint64_t L[R];
#pragma unroll
    for (int r = 0; r < R; ++r) L[r] = KEY_INF;
    for (uint32_t t = prefix[q]; t < prefix[q + 1]; ++t) {
        uint64_t B[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = r * 32 + lane;
            B[r] = e < ntop ? partial[(int64_t)t * ntop + e] : KEY_INF;
        }
        merge_sorted<R>(L, B);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = r * 32 + lane;
        if (e < ntop) topkeys[q * ntop + e] = L[r];
    }
}

void launch_tile_plan(const DeviceIndex &ix, const int32_t *probes, const int32_t *npq, int64_t nq,
                      int32_t nprobe, int32_t stride, uint32_t T_req, uint32_t cap,
                      uint32_t *chunks, unsigned long long *total, uint32_t *T_out,
                      uint32_t *prefix, cudaStream_t st) {
    FA_CHECK_CUDA(cudaMemsetAsync(total, 0, sizeof(unsigned long long), st));
    k_tile_count<<<(unsigned)((nq + 7) / 8), 256, 0, st>>>(probes, npq, nq, nprobe, stride,
                                                            ix.list_beg, ix.rep_off, ix.nlist,
                                                            ix.n_rep > 0, chunks, total);
    k_tile_plan<<<1, 1024, 0, st>>>(chunks, nq, T_req, cap, total, T_out, prefix);
    FA_CHECK_CUDA(cudaGetLastError());
}

void launch_tile_merge(const uint64_t *partial, const uint32_t *prefix, int64_t nq, int32_t ntop,
                       uint64_t *topkeys, cudaStream_t st) {
    const dim3 grid((unsigned)((nq + 7) / 8));
    if (ntop <= 32) k_tile_merge<1><<<grid, 256, 0, st>>>(partial, prefix, nq, ntop, topkeys);
    else if (ntop <= 64) k_tile_merge<2><<<grid, 256, 0, st>>>(partial, prefix, nq, ntop, topkeys);
    else if (ntop <= 128) k_tile_merge<4><<<grid, 256, 0, st>>>(partial, prefix, nq, ntop, topkeys);
    else k_tile_merge<8><<<grid, 256, 0, st>>>(partial, prefix, nq, ntop, topkeys);
    FA_CHECK_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Processing order: queries bucketed by their nearest (first) probed list.
// Counting sort: histogram, exclusive scan, scatter. The order inside a
// bucket depends on atomics, which does not matter: every query is scanned
// whole by one CTA, whatever its slot.
// ---------------------------------------------------------------------------
__global__ void k_order_hist(const int32_t *probes, int64_t nq, int32_t stride, int32_t nlist,
                             uint32_t *cnt) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int l = probes[q * stride];
        atomicAdd(&cnt[(l >= 0 && l < nlist) ? l : 0], 1u);
    }
}

__global__ void k_order_scan(uint32_t *cnt, int32_t nlist) {
    // one CTA of 1024 threads: exclusive scan in place, chunk by chunk
    __shared__ uint32_t part[32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nlist; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nlist ? cnt[i] : 0u;
        uint32_t inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) part[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            uint32_t p = lane < (int)(blockDim.x >> 5) ? part[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, p, o);
                if (lane >= o) p += y;
            }
            part[lane] = p;
        }
        __syncthreads();
        const uint32_t excl = carry + (warp ? part[warp - 1] : 0u) + inc - v;
        if (i < nlist) cnt[i] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
}

__global__ void k_order_scatter(const int32_t *probes, int64_t nq, int32_t stride, int32_t nlist,
                                uint32_t *off, int32_t *order) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int l = probes[q * stride];
        const uint32_t p = atomicAdd(&off[(l >= 0 && l < nlist) ? l : 0], 1u);
        order[p] = (int32_t)q;
    }
}

void launch_query_order(const int32_t *probes, int64_t nq, int32_t stride, int32_t nlist,
                        uint32_t *cnt, int32_t *order, cudaStream_t st) {
    if (nq == 0) return;
    FA_CHECK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)nlist, st));
    const int grid = (int)std::min<int64_t>((nq + 255) / 256, 4096);
    k_order_hist<<<grid, 256, 0, st>>>(probes, nq, stride, nlist, cnt);
    k_order_scan<<<1, 1024, 0, st>>>(cnt, nlist);
    k_order_scatter<<<grid, 256, 0, st>>>(probes, nq, stride, nlist, cnt, order);
    FA_CHECK_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Test hook: the distinct ids of one query as the scan's dedup rule keeps them
// (internal ids, unordered), one warp per segment.
// ---------------------------------------------------------------------------
__global__ void k_debug_candidates(const uint32_t *list_beg, const uint64_t *rep_off,
                                   const uint32_t *rep_v, const uint32_t *rep_mo,
                                   const uint8_t *rep_t, const uint32_t *mem, int32_t nlist,
                                   int32_t has_rep, const int32_t *probes, int32_t np,
                                   uint32_t *out, uint32_t *count, uint32_t cap, uint32_t *err) {
    extern __shared__ uint32_t bm[];
    const int nw = (nlist + 31) / 32;
    for (int j = threadIdx.x; j < nw; j += blockDim.x) bm[j] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const int l = probes[i];
        if (l >= 0 && l < nlist) atomicOr(&bm[l >> 5], 1u << (l & 31));
    }
    __syncthreads();
    for (int i = 0; i < np; ++i) {
        const int l = probes[i];
        if (l < 0 || l >= nlist) continue;
        for (uint32_t v = list_beg[l] + threadIdx.x; v < list_beg[l + 1]; v += blockDim.x) {
            const uint32_t p = atomicAdd(count, 1u);
            if (p < cap) out[p] = v;
            else atomicOr(err, DEV_ERR_OVERFLOW);
        }
        if (!has_rep) continue;
        for (uint64_t e = rep_off[l] + threadIdx.x; e < rep_off[l + 1]; e += blockDim.x) {
            bool keep = true;
            for (int u = 0; u < rep_t[e]; ++u) {
                const uint32_t ll = mem[rep_mo[e] + u];
                if (bm[ll >> 5] & (1u << (ll & 31))) keep = false;
            }
            if (keep) {
                const uint32_t p = atomicAdd(count, 1u);
                if (p < cap) out[p] = rep_v[e];
                else atomicOr(err, DEV_ERR_OVERFLOW);
            }
        }
    }
}

void launch_debug_candidates(const DeviceIndex &ix, const int32_t *probes, int32_t np,
                             uint32_t *out, uint32_t *count, uint32_t cap, cudaStream_t st) {
    const int smem = ((ix.nlist + 31) / 32) * 4;
    FA_CHECK_CUDA(cudaFuncSetAttribute(k_debug_candidates,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_debug_candidates<<<1, 256, smem, st>>>(ix.list_beg, ix.rep_off, ix.rep_v, ix.rep_mo,
                                             ix.rep_t, ix.mem, ix.nlist, ix.n_rep > 0, probes,
                                             np, out, count, cap, count + 1);
    FA_CHECK_CUDA(cudaGetLastError());
}

}  // namespace fa
