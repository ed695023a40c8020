// Steps 1 and 3-7 of the filtering path for one query per CTA:
//   LUT (step 1)       dist(q_i, c) for the M subspaces, into shared memory
//   gather (3-4)       the probed lists' primary ranges and replica slices
//   dedup (5)          each distinct vector once (probe-set rule below)
//   ADC (6, Eq. 1)     dist(q, v) = sum_i LUT[i][code_i(v)], FP32
//   top-n (7)          per-warp running selection, merged per CTA
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

#include "../fa_internal.h"
#include "warp_topk.cuh"

namespace fa {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_WARPS = SCAN_THREADS / 32;
constexpr int MAX_PROBE = 512;
constexpr int MAX_D = 1024;

struct ScanArgs {
    // index
    const uint8_t *codes;
    const uint32_t *list_beg;
    const uint64_t *rep_off;
    const uint32_t *rep_v, *rep_mo;
    const uint8_t *rep_t;
    const uint32_t *mem;
    const float *codebooks;
    int32_t d, M, dsub, nlist;
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
};

// Shared memory plan (bytes), shared by host and device.
struct ScanSmem {
    int lut, qv, seg, bitmap, wbuf, total, npmax;
    __host__ __device__ ScanSmem(int M, int W, int d, int nlist, int has_rep, int nprobe) {
        (void)M;
        npmax = nprobe;
        lut = 256 * W * 4;
        qv = ((d + 3) & ~3) * 4;
        seg = ((2 * nprobe + 1) * 4 + 15) / 16 * 16 /*pref*/ + 2 * nprobe * 4 * 2 /*beg,end*/;
        bitmap = has_rep ? ((nlist + 127) / 128) * 16 : 0;
        wbuf = SCAN_WARPS * 64 * 8;
        total = lut + qv + seg + bitmap + wbuf;
    }
};

__device__ __forceinline__ float lut_entry_global(const ScanArgs &a, int64_t qi, int m, int c) {
    const int64_t base = qi * (int64_t)a.M * 256 + (int64_t)m * 256 + c;
    const float *sc = a.lut_scale + qi * (2 + a.M);
    if (a.lut_prec == FA_LUT_F32) return reinterpret_cast<const float *>(a.lut)[base];
    if (a.lut_prec == FA_LUT_F16)
        return __half2float(reinterpret_cast<const __half *>(a.lut)[base]) * sc[0] + sc[2 + m];
    __nv_fp8_e4m3 v;
    v.__x = reinterpret_cast<const uint8_t *>(a.lut)[base];
    return float(v) * sc[0] + sc[2 + m];
}

// Builds the LUT of query qi in shared memory (rows of W floats).
template <int W>
__device__ __forceinline__ void build_lut(const ScanArgs &a, int64_t qi, float *lut, const float *qv) {
    const int M = a.M, dsub = a.dsub;
    const int P = M + 31;  // positions used per row
    for (int idx = threadIdx.x; idx < 256 * M; idx += blockDim.x) {
        const int c = idx / M, m = idx - c * M;
        float val;
        if (a.lut_prec < 0) {
            const float *cw = a.codebooks + ((int64_t)m * 256 + c) * dsub;
            const float *qm = qv + m * dsub;
            float s = 0.f;
            for (int j = 0; j < dsub; ++j) {
                const float t = qm[j] - cw[j];
                s = fmaf(t, t, s);
            }
            val = s;
        } else {
            val = lut_entry_global(a, qi, m, c);
        }
        for (int p = m; p < P; p += M) lut[c * W + p] = val;
    }
}

// ADC distance of one code row (rotation r = v mod 32) against the smem LUT.
template <int M, int W>
__device__ __forceinline__ float adc_row(const uint8_t *row, uint32_t v, const float *lut, bool valid) {
    constexpr int NW = M / 4;
    uint32_t w[NW];
    if (valid) {
        if (M % 16 == 0) {
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
        for (int i = 0; i < NW; ++i) w[i] = 0;
    }
    const uint32_t r4 = (v & 31u) * 4u;
    const char *lb = reinterpret_cast<const char *>(lut);
    float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
    for (int s = 0; s < M; ++s) {
        uint32_t off;
        if (W == 64) {
            // (code << 8) | r4 in one byte permute: byte0 <- r4, byte1 <- code
            off = __byte_perm(w[s >> 2], r4, 0x5504u | ((uint32_t)(s & 3) << 4));
        } else {
            const uint32_t c = __byte_perm(w[s >> 2], 0u, 0x4440u | (uint32_t)(s & 3));
            off = c * (uint32_t)(W * 4) + r4;
        }
        const float x = *reinterpret_cast<const float *>(lb + off + 4 * s);
        if (s & 1)
            acc1 += x;
        else
            acc0 += x;
    }
    return acc0 + acc1;
}

template <int M, int W, int R>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan(const ScanArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const ScanSmem plan(M, W, a.d, a.nlist, a.has_rep, a.nprobe);
    float *lut = reinterpret_cast<float *>(smem);
    float *qv = reinterpret_cast<float *>(smem + plan.lut);
    uint32_t *pref = reinterpret_cast<uint32_t *>(smem + plan.lut + plan.qv);
    uint32_t *seg_beg = reinterpret_cast<uint32_t *>(smem + plan.lut + plan.qv +
                                                     ((2 * a.nprobe + 1) * 4 + 15) / 16 * 16);
    uint32_t *seg_end = seg_beg + 2 * a.nprobe;
    uint32_t *bitmap = reinterpret_cast<uint32_t *>(smem + plan.lut + plan.qv + plan.seg);
    uint64_t *wbuf = reinterpret_cast<uint64_t *>(smem + plan.lut + plan.qv + plan.seg + plan.bitmap);
    __shared__ int64_t s_q;
    __shared__ uint32_t s_kept;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int64_t it = 0;; ++it) {
        if (threadIdx.x == 0) {
            if (a.persistent)
                s_q = (int64_t)atomicAdd(a.tile_ctr, 1u);
            else
                s_q = (int64_t)blockIdx.x + it * gridDim.x;
            s_kept = 0;
        }
        __syncthreads();
        const int64_t qi = s_q;
        if (qi >= a.nq) break;

        int np = a.npq ? a.npq[qi] : a.nprobe;
        np = np < 1 ? 1 : (np > a.nprobe ? a.nprobe : np);
        const int ntop = a.ntopq ? a.ntopq[qi] : a.ntop;
        const int32_t *pr = a.probes + qi * a.probe_stride;

        // query, segment bounds, probed-list bitmap
        for (int j = threadIdx.x; j < a.d; j += blockDim.x) qv[j] = a.q[qi * a.d + j];
        if (a.has_rep)
            for (int j = threadIdx.x; j < (a.nlist + 31) / 32; j += blockDim.x) bitmap[j] = 0u;
        for (int i = threadIdx.x; i < np; i += blockDim.x) {
            int l = pr[i];
            if (l < 0 || l >= a.nlist) {
                atomicOr(a.err, DEV_ERR_BOUNDS);
                l = 0;
                seg_beg[i] = seg_end[i] = 0;
                seg_beg[np + i] = seg_end[np + i] = 0;
                continue;
            }
            seg_beg[i] = a.list_beg[l];
            seg_end[i] = a.list_beg[l + 1];
            if (a.has_rep) {
                seg_beg[np + i] = (uint32_t)a.rep_off[l];
                seg_end[np + i] = (uint32_t)a.rep_off[l + 1];
            } else {
                seg_beg[np + i] = seg_end[np + i] = 0;
            }
        }
        __syncthreads();
        if (a.has_rep)
            for (int i = threadIdx.x; i < np; i += blockDim.x) {
                const int l = pr[i];
                if (l >= 0 && l < a.nlist) atomicOr(&bitmap[l >> 5], 1u << (l & 31));
            }
        // chunk prefix over 2*np segments (warp 0)
        if (warp == 0) {
            const int nseg = 2 * np;
            const int per = (nseg + 31) / 32;
            uint32_t loc = 0;
            for (int t = 0; t < per; ++t) {
                const int s = lane * per + t;
                if (s < nseg) loc += (seg_end[s] - seg_beg[s] + 31u) >> 5;
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
                    pref[s] = run;
                    run += (seg_end[s] - seg_beg[s] + 31u) >> 5;
                }
            }
            if (lane == 31) pref[nseg] = inc;
        }
        build_lut<W>(a, qi, lut, qv);
        __syncthreads();

        // scan
        WarpTopK<R> tk;
        tk.init(wbuf + warp * 64, ntop);
        const int nseg = 2 * np;
        const uint32_t total = pref[nseg];
        uint32_t kept = 0;
        int sg = 0;
        for (uint32_t g = warp; g < total; g += SCAN_WARPS) {
            while (g >= pref[sg + 1]) ++sg;
            const uint32_t pos = seg_beg[sg] + ((g - pref[sg]) << 5) + lane;
            bool valid = pos < seg_end[sg];
            uint32_t v = pos;
            if (sg >= np && valid) {
                // replica entry: scanned only if no earlier list of v is probed
                v = a.rep_v[pos];
                const uint32_t mo = a.rep_mo[pos];
                const int t = a.rep_t[pos];
                for (int u = 0; u < t; ++u) {
                    const uint32_t l = a.mem[mo + u];
                    if (bitmap[l >> 5] & (1u << (l & 31))) valid = false;
                }
            }
            const float dist = adc_row<M, W>(a.codes + (size_t)v * M, v, lut, valid);
            kept += valid ? 1u : 0u;
            tk.push(make_key(dist, v), valid);
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
            for (int w = 1; w < SCAN_WARPS; ++w) {
                uint64_t B[R];
#pragma unroll
                for (int r = 0; r < R; ++r) B[r] = mrg[w * 32 * R + r * 32 + lane];
                merge_sorted<R>(L, B);
            }
            uint64_t *out = a.topkeys + qi * (int64_t)a.ntop;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int e = r * 32 + lane;
                if (e < a.ntop) out[e] = e < ntop ? L[r] : KEY_INF;
            }
            if (a.stats && lane == 0) {
                int64_t gathered = 0;
                for (int s = 0; s < np; ++s) gathered += seg_end[s] - seg_beg[s];
                for (int s = np; s < 2 * np; ++s) gathered += seg_end[s] - seg_beg[s];
                a.stats[qi * 4 + 0] = (int32_t)gathered;
                a.stats[qi * 4 + 1] = (int32_t)s_kept;
            }
        }
        __syncthreads();
    }
}

template <int M, int W, int R>
static void launch_scan_t(const ScanArgs &a, int smem_bytes, int grid, cudaStream_t st) {
    auto kfn = k_scan<M, W, R>;
    FA_CHECK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes));
    kfn<<<grid, SCAN_THREADS, smem_bytes, st>>>(a);
    FA_CHECK_CUDA(cudaGetLastError());
}

template <int M, int W>
static void launch_scan_r(const ScanArgs &a, int smem, int grid, cudaStream_t st) {
    if (a.ntop <= 32)
        launch_scan_t<M, W, 1>(a, smem, grid, st);
    else if (a.ntop <= 64)
        launch_scan_t<M, W, 2>(a, smem, grid, st);
    else if (a.ntop <= 128)
        launch_scan_t<M, W, 4>(a, smem, grid, st);
    else
        launch_scan_t<M, W, 8>(a, smem, grid, st);
}

void launch_scan(const DeviceIndex &ix, const ScanLaunch &l, cudaStream_t st) {
    if (l.nq == 0) return;
    FA_REQUIRE(l.nprobe <= MAX_PROBE, FA_ERR_ARG, "nprobe above 512");
    FA_REQUIRE(ix.d <= MAX_D, FA_ERR_ARG, "d above 1024");
    FA_REQUIRE(l.ntop >= 1 && l.ntop <= 256, FA_ERR_ARG, "top-n must be in 1..256");
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
    a.M = ix.M;
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
    const int W = lut_row_words(ix.M);
    const ScanSmem plan(ix.M, W, ix.d, ix.nlist, a.has_rep, l.nprobe);
    // the merge area reuses the LUT region: SCAN_WARPS * 32R keys
    FA_REQUIRE(SCAN_WARPS * 256 * 8 <= plan.lut, FA_ERR_ARG, "LUT region too small for merge");
    FA_REQUIRE(plan.total <= 227 * 1024, FA_ERR_ARG, "scan shared memory above 227 KB");
    int grid;
    if (l.persistent) {
        int per_sm = (227 * 1024) / (plan.total + 1024);
        if (per_sm < 1) per_sm = 1;
        if (per_sm > 8) per_sm = 8;
        grid = num_sms(0) * per_sm;
        if ((int64_t)grid > l.nq) grid = (int)l.nq;
    } else {
        grid = (int)(l.nq < (int64_t)INT32_MAX ? l.nq : INT32_MAX);
    }
    switch (ix.M) {
        case 8: launch_scan_r<8, 64>(a, plan.total, grid, st); break;
        case 16: launch_scan_r<16, 64>(a, plan.total, grid, st); break;
        case 32: launch_scan_r<32, 64>(a, plan.total, grid, st); break;
        case 48: launch_scan_r<48, 80>(a, plan.total, grid, st); break;
        case 64: launch_scan_r<64, 128>(a, plan.total, grid, st); break;
        default: FA_REQUIRE(false, FA_ERR_ARG, "M must be one of 8, 16, 32, 48, 64");
    }
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
