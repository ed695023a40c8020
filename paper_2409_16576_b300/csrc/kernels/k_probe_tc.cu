// Coarse probe (step 2) as one fused tensor-core kernel: distances of a tile
// of 128 queries to every centroid, and each query's nprobe nearest lists,
// without writing the query x centroid distance matrix.
//
//   d2(q, c_l) = |q|^2 - 2 q.c_l + |c_l|^2
//
// The dot products run on the tensor cores exactly as in the unfused form:
// queries and centroids split into bf16 pairs hi + lo, three MMAs per K-step
// (hi.hi + hi.lo + lo.hi), FP32 accumulation in tensor memory.
//
// Work: the (query tile, 128-centroid tile) pairs are laid out query-tile
// major and cut into one contiguous range per CTA, so every SM gets the same
// number of MMA tiles; a CTA whose range crosses into the next query tile
// reloads its queries there. Within a range:
//   - thread 0 streams centroid tiles into a two-stage shared-memory ring with
//     bulk copies (mbarrier completion) and issues the MMAs of tile i into one
//     of two tensor-memory accumulators;
//   - meanwhile all 8 warps run the epilogue of tile i-1 from the other
//     accumulator. Warps w and w+4 read the same 32 TMEM lanes (queries) and
//     split the 128 columns in halves.
// Selection: each (query, column half) appends the keys (distance, list id)
// below the query's threshold to a private queue in global memory. A full
// queue is cut back to its n smallest by the warp together (the bitonic top-n
// of warp_topk.cuh); its n-th smallest then bounds the query's threshold,
// which the two halves share in shared memory. At the end of a range every queue holds its n
// smallest keys, sorted; k_probe_merge takes each query's n smallest over its
// queues. Keys order by (distance, list id), so the result is the same set
// and order as a full sort of the distance row.
#include <algorithm>

#include "../fa_internal.h"
#include "tc_util.cuh"
#include "warp_topk.cuh"

namespace fa {

namespace {

constexpr int PQ = 128;  // queries per tile (MMA M = tensor-memory lanes)
constexpr int PN = 128;  // centroids per tile (MMA N)
constexpr int PT = 256;  // 8 warps: two per lane quadrant, one column half each
constexpr uint32_t PWAIT = 1u << 22;

struct ProbeArgs {
    const float *q;              // [rows][d]
    int64_t rows;
    int32_t d, Kp;
    const __nv_bfloat16 *tiles;  // 256-centroid tiles [T][hi, lo][256 * Kp], core-matrix layout
    const float *cnorm;          // [nlist] |c|^2
    int32_t nlist;
    int32_t nt;                  // 128-centroid tiles
    int64_t total;               // query tiles * nt
    int32_t per;                 // (query tile, centroid tile) pairs per CTA
    int32_t segmax;              // queue sets per query
    int32_t cap;                 // queue capacity (keys)
    int32_t n;                   // lists wanted per query
    uint64_t *lists;             // [rows][segmax][2][cap]
    uint32_t *err;
};

// Cuts the queue of lane `src` back to its n smallest keys, sorted and padded
// with KEY_INF to n. The queue is its sorted part [0, nsorted) followed by the
// keys appended since [nsorted, cnt); both are loaded at once, the sorted part
// straight into the top-n registers, and only the new keys are merged. The
// new n-th smallest tightens the query's shared threshold.
template <int R>
__device__ __forceinline__ void compact(uint64_t *myq, int &cnt, int &nsorted,
                                        unsigned long long *tsh, int src, int n, uint64_t *wbuf) {
    const int lane = threadIdx.x & 31;
    uint64_t *base = reinterpret_cast<uint64_t *>(shfl64(reinterpret_cast<uint64_t>(myq), src));
    const int c = __shfl_sync(FULL, cnt, src);
    const int ns = __shfl_sync(FULL, nsorted, src);
    __syncwarp();
    WarpTopK<R> tk;
    tk.init(wbuf, n);
    uint64_t nk[R + 2];  // c - ns <= 32 R + 64 new keys
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = r * 32 + lane;
        tk.L[r] = e < ns ? base[e] : KEY_INF;
    }
#pragma unroll
    for (int b = 0; b < R + 2; ++b) {
        const int e = ns + b * 32 + lane;
        nk[b] = e < c ? base[e] : KEY_INF;
    }
    if (ns >= n) tk.thr = warp_elem<R>(tk.L, n - 1);
#pragma unroll
    for (int b = 0; b < R + 2; ++b)
        if (ns + b * 32 < c) tk.push(nk[b], ns + b * 32 + lane < c);
    tk.finish();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = r * 32 + lane;
        if (e < n) base[e] = tk.L[r];
    }
    const uint64_t kth = warp_elem<R>(tk.L, n - 1);
    if (lane == 0 && kth != KEY_INF) atomicMin(tsh + src, (unsigned long long)kth);
    __syncwarp();
    if (lane == src) cnt = nsorted = c < n ? c : n;
}

template <int R>
__global__ void __launch_bounds__(PT, 1) k_probe_tc(const ProbeArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t full[2], mdone[2];
    __shared__ uint32_t tmem_base;
    __shared__ uint64_t wbuf[PT / 32][64];
    // per query of the tile: the smallest n-th-smallest key over its two queues;
    // no key at or above it can be among the query's n nearest lists
    __shared__ unsigned long long tau_sh[PQ];
    const int Kp = a.Kp;
    const uint32_t half_bytes = (uint32_t)PN * Kp * 2;  // hi (or lo) of one 128-centroid tile
    __nv_bfloat16 *Ahi = reinterpret_cast<__nv_bfloat16 *>(sm);
    __nv_bfloat16 *Alo = Ahi + PQ * Kp;
    unsigned char *Bs = sm + (size_t)2 * PQ * Kp * 2;  // 2 stages x (hi, lo)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, colh = warp >> 2;
    const int64_t g0 = (int64_t)blockIdx.x * a.per;
    const int64_t g1 = min(a.total, g0 + a.per);
    if (g0 >= g1) return;

    if (warp == 0) tc::tmem_alloc(&tmem_base, 2 * PN);
    if (tid == 0) {
        tc::mbar_init(&full[0], 1);
        tc::mbar_init(&full[1], 1);
        tc::mbar_init(&mdone[0], 1);
        tc::mbar_init(&mdone[1], 1);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = tmem_base;
    const uint32_t idesc = tc::idesc_bf16_f32(PQ, PN);
    const uint32_t sbo = (uint32_t)(Kp / 8) * 128u;
    const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo);
    // bit s: phase parity to wait for next on full[s] / mdone[s]; copies and
    // MMAs in flight (thread 0's view), kept as bit masks so nothing is indexed
    // at run time
    uint32_t fph = 0u, mph = 0u, lpend = 0u, mpend = 0u;
    bool failed = false;

    auto issue_load = [&](int s, int64_t gi) {
        const int t128 = (int)(gi % a.nt);
        const __nv_bfloat16 *hi = a.tiles + (size_t)(t128 >> 1) * 2 * 256 * Kp + (size_t)(t128 & 1) * PN * Kp;
        const __nv_bfloat16 *lo = hi + (size_t)256 * Kp;
        unsigned char *dst = Bs + (size_t)s * 2 * half_bytes;
        tc::mbar_expect_tx(&full[s], 2 * half_bytes);
        tc::bulk_g2s(dst, hi, half_bytes, &full[s]);
        tc::bulk_g2s(dst + half_bytes, lo, half_bytes, &full[s]);
        lpend |= 1u << s;
    };

    int64_t g = g0;
    while (g < g1 && !failed) {
        const int64_t qt = g / a.nt;
        const int64_t s_end = min(g1, (qt + 1) * a.nt);
        const int nseg = (int)(s_end - g);
        const int seg = (int)(blockIdx.x - (qt * a.nt) / a.per);
        const int64_t r0 = qt * PQ;
        // A: this query tile as bf16 hi/lo (every MMA on the previous tile is done)
        for (int e = tid; e < PQ * Kp; e += PT) {
            const int r = e / Kp, k = e - r * Kp;
            const float x = (r0 + r < a.rows && k < a.d) ? a.q[(r0 + r) * a.d + k] : 0.f;
            __nv_bfloat16 h, l;
            tc::split_bf16(x, h, l);
            const uint32_t o = tc::core_offset(r, k, Kp) >> 1;
            Ahi[o] = h;
            Alo[o] = l;
        }
        const int64_t row = r0 + quad * 32 + lane;
        const bool rv = row < a.rows;
        float qn = 0.f;
        if (rv)
            for (int k = 0; k < a.d; ++k) {
                const float x = a.q[row * a.d + k];
                qn = fmaf(x, x, qn);
            }
        uint64_t *myq = rv ? a.lists + (((size_t)row * a.segmax + seg) * 2 + colh) * a.cap : nullptr;
        unsigned long long *tsh = tau_sh + quad * 32;
        int cnt = 0, nsorted = 0;
        if (tid < PQ) tau_sh[tid] = KEY_INF;
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            issue_load(0, g);
            if (nseg > 1) issue_load(1, g + 1);
        }
        for (int i = 0; i <= nseg; ++i) {
            bool ok = true;
            if (i < nseg && tid == 0) {
                const int s = i & 1;
                ok = tc::mbar_wait(&full[s], (fph >> s) & 1u, PWAIT);
                if (ok) {
                    fph ^= 1u << s;
                    lpend &= ~(1u << s);
                    tc::fence_after();
                    const uint32_t bh = tc::smem_u32(Bs + (size_t)s * 2 * half_bytes), bl = bh + half_bytes;
                    const uint32_t acc = tbase + (uint32_t)(i & 1) * PN;
                    for (int ks = 0; ks < Kp / 16; ++ks) {
                        const uint32_t off = 256u * ks;
                        const uint64_t dah = tc::smem_desc(ah + off, 128, sbo);
                        const uint64_t dal = tc::smem_desc(al + off, 128, sbo);
                        const uint64_t dbh = tc::smem_desc(bh + off, 128, sbo);
                        const uint64_t dbl = tc::smem_desc(bl + off, 128, sbo);
                        tc::mma_bf16(acc, dah, dbh, idesc, ks > 0 ? 1u : 0u);
                        tc::mma_bf16(acc, dah, dbl, idesc, 1u);
                        tc::mma_bf16(acc, dal, dbh, idesc, 1u);
                    }
                    tc::mma_commit(&mdone[i & 1]);
                    mpend |= 1u << (i & 1);
                }
            }
            if (i >= 1) {
                const int b = (i - 1) & 1;
                ok = ok && tc::mbar_wait(&mdone[b], (mph >> b) & 1u, PWAIT);
                if (ok) {
                    mph ^= 1u << b;
                    mpend &= ~(1u << b);
                }
            }
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            if (i == 0) continue;
            // tile j = i - 1: its MMAs are done, so its stage takes tile j + 2
            const int j = i - 1, b = j & 1;
            tc::fence_after();
            if (tid == 0 && j + 2 < nseg) issue_load(b, g + j + 2);
            const int lbase = (int)((g + j) % a.nt) * PN + colh * 64;
            const uint32_t taddr = tbase + ((uint32_t)(quad * 32) << 16) + (uint32_t)b * PN + colh * 64;
#pragma unroll 1
            for (int c0 = 0; c0 < 64; c0 += 32) {
                float v[32];
                tc::tmem_ld32(taddr + c0, v);
                uint32_t need = __ballot_sync(FULL, rv && cnt + 32 > a.cap);
                while (need) {
                    const int src = __ffs(need) - 1;
                    compact<R>(myq, cnt, nsorted, tsh, src, a.n, wbuf[warp]);
                    need &= need - 1;
                }
                const uint64_t tau = *reinterpret_cast<volatile unsigned long long *>(tsh + lane);
                const float tau_d = tau == KEY_INF ? INFINITY : o2f((uint32_t)(tau >> 32));
                if (rv) {
                    const int l0 = lbase + c0;
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        const int l = l0 + e;
                        if (l < a.nlist) {
                            const float dd = qn - 2.f * v[e] + __ldg(a.cnorm + l);
                            if (dd <= tau_d) {
                                const uint64_t key = make_key(dd, (uint32_t)l);
                                if (key < tau) myq[cnt++] = key;
                            }
                        }
                    }
                }
            }
            tc::fence_before();
            __syncthreads();
        }
        if (failed) break;
        // every queue of this range down to its sorted n smallest
        uint32_t m = __ballot_sync(FULL, rv);
        while (m) {
            const int src = __ffs(m) - 1;
            compact<R>(myq, cnt, nsorted, tsh, src, a.n, wbuf[warp]);
            m &= m - 1;
        }
        // the thresholds are reset for the next query tile only after every warp is done
        __syncthreads();
        g = s_end;
    }
    if (failed && tid == 0) {
        atomicOr(a.err, DEV_ERR_TIMEOUT);
        // copies and MMAs still in flight finish before shared and tensor memory go
        for (int s = 0; s < 2; ++s)
            if ((lpend >> s) & 1u) tc::mbar_wait(&full[s], (fph >> s) & 1u, PWAIT);
        for (int b = 0; b < 2; ++b)
            if ((mpend >> b) & 1u) tc::mbar_wait(&mdone[b], (mph >> b) & 1u, PWAIT);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_free(tbase, 2 * PN);
}

// One warp per query: the n smallest keys over the query's sorted queues.
template <int R>
__global__ void __launch_bounds__(256) k_probe_merge(const uint64_t *__restrict__ lists, int64_t rows,
                                                     int32_t nt, int32_t per, int32_t segmax,
                                                     int32_t cap, int32_t n,
                                                     int32_t *__restrict__ out_ids,
                                                     int32_t out_stride) {
    __shared__ uint64_t wbuf[8][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * 8 + warp;
    if (row >= rows) return;
    const int64_t qt = row / PQ;
    const int64_t c0 = qt * nt / per, c1 = ((qt + 1) * nt - 1) / per;
    const int ns = (int)(c1 - c0 + 1);
    WarpTopK<R> tk;
    tk.init(wbuf[warp], n);
    for (int s = 0; s < ns; ++s)
        for (int h = 0; h < 2; ++h) {
            const uint64_t *L = lists + (((size_t)row * segmax + s) * 2 + h) * cap;
            for (int o = 0; o < n; o += 32) {
                const bool ok = o + lane < n;
                tk.push(ok ? L[o + lane] : KEY_INF, ok);
            }
        }
    tk.finish();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = r * 32 + lane;
        if (e < n) {
            const uint64_t k = tk.L[r];
            out_ids[row * out_stride + e] = k == KEY_INF ? -1 : (int32_t)(k & 0xffffffffu);
        }
    }
}

struct ProbePlan {
    int32_t nt, per, grid, segmax, cap, R;
    int64_t total;
    size_t bytes;
};

ProbePlan probe_plan(int32_t nlist, int64_t nq, int32_t ntop) {
    ProbePlan p{};
    p.nt = (nlist + PN - 1) / PN;
    const int64_t qtiles = (nq + PQ - 1) / PQ;
    p.total = qtiles * p.nt;
    p.per = (int32_t)((p.total + num_sms(0) - 1) / num_sms(0));
    p.grid = (int32_t)((p.total + p.per - 1) / p.per);
    p.segmax = std::min<int32_t>(p.grid, (p.nt + p.per - 1) / p.per + 1);
    p.R = ntop <= 32 ? 1 : ntop <= 64 ? 2 : ntop <= 128 ? 4 : ntop <= 256 ? 8 : 16;
    p.cap = 32 * p.R + 64;
    p.bytes = (size_t)nq * p.segmax * 2 * p.cap * sizeof(uint64_t);
    return p;
}

template <int R>
void launch_r(const ProbeArgs &a, const ProbePlan &p, int smem, int32_t *probes, int32_t stride,
              cudaStream_t st) {
    FA_CHECK_CUDA(cudaFuncSetAttribute(k_probe_tc<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_probe_tc<R><<<p.grid, PT, smem, st>>>(a);
    FA_CHECK_CUDA(cudaGetLastError());
    k_probe_merge<R><<<(unsigned)((a.rows + 7) / 8), 256, 0, st>>>(a.lists, a.rows, p.nt, p.per, p.segmax,
                                                                   p.cap, a.n, probes, stride);
    FA_CHECK_CUDA(cudaGetLastError());
}

}  // namespace

size_t probe_tc_scratch_bytes(const DeviceIndex &ix, int64_t nq, int32_t ntop) {
    if (nq <= 0 || !ix.centroids_bf16) return 0;
    return probe_plan(ix.nlist, nq, ntop).bytes;
}

void launch_probe_tc(const DeviceIndex &ix, const float *q, int64_t nq, int32_t ntop, int32_t *probes,
                     int32_t probe_stride, uint64_t *scratch, size_t scratch_bytes, uint32_t *err,
                     cudaStream_t st) {
    if (nq == 0) return;
    FA_REQUIRE(ix.centroids_bf16 != nullptr, FA_ERR_ARG, "tensor-core centroid tiles missing");
    FA_REQUIRE(ntop >= 1 && ntop <= 512, FA_ERR_ARG, "top-n of the coarse probe must be in 1..512");
    const ProbePlan p = probe_plan(ix.nlist, nq, ntop);
    FA_REQUIRE(scratch && scratch_bytes >= p.bytes, FA_ERR_STATE, "probe scratch too small");
    ProbeArgs a{};
    a.q = q;
    a.rows = nq;
    a.d = ix.d;
    a.Kp = ix.tc_kp;
    a.tiles = reinterpret_cast<const __nv_bfloat16 *>(ix.centroids_bf16);
    a.cnorm = ix.cnorm;
    a.nlist = ix.nlist;
    a.nt = p.nt;
    a.total = p.total;
    a.per = p.per;
    a.segmax = p.segmax;
    a.cap = p.cap;
    a.n = ntop;
    a.lists = scratch;
    a.err = err;
    // queries + two centroid stages; at least 116 KB so that one CTA (256 TMEM
    // columns) runs per SM and tensor-memory allocation never waits
    const int smem = std::max(3 * 2 * PQ * a.Kp * 2, 116 * 1024);
    FA_REQUIRE(a.Kp <= 128, FA_ERR_ARG, "tensor-core coarse probe supports d <= 128");
    switch (p.R) {
        case 1: launch_r<1>(a, p, smem, probes, probe_stride, st); break;
        case 2: launch_r<2>(a, p, smem, probes, probe_stride, st); break;
        case 4: launch_r<4>(a, p, smem, probes, probe_stride, st); break;
        case 8: launch_r<8>(a, p, smem, probes, probe_stride, st); break;
        default: launch_r<16>(a, p, smem, probes, probe_stride, st); break;
    }
}

}  // namespace fa
