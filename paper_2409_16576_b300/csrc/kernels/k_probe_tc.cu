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
    unsigned long long *gtau;    // [rows] per-query threshold shared by the CTAs on its tile
    uint32_t *err;
};

// Cuts the queue of lane `src` back to its n smallest keys, sorted and padded
// with KEY_INF to n. The queue is its sorted part [0, nsorted) followed by the
// keys appended since [nsorted, cnt); both are loaded at once, the sorted part
// straight into the top-n registers, and only the new keys are merged. The
// new n-th smallest tightens the query's shared threshold.
template <int R>
__device__ __forceinline__ void compact(uint64_t *myq, int &cnt, int &nsorted,
                                        unsigned long long *tsh, unsigned long long *gt, int src,
                                        int n, uint64_t *wbuf) {
    const int lane = threadIdx.x & 31;
    uint64_t *base = reinterpret_cast<uint64_t *>(shfl64(reinterpret_cast<uint64_t>(myq), src));
    unsigned long long *gsrc =
        reinterpret_cast<unsigned long long *>(shfl64(reinterpret_cast<uint64_t>(gt), src));
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
    if (lane == 0 && kth != KEY_INF) {
        atomicMin(tsh + src, (unsigned long long)kth);
        atomicMin(gsrc, (unsigned long long)kth);
    }
    __syncwarp();
    if (lane == src) cnt = nsorted = c < n ? c : n;
}

template <int R>
__global__ void __launch_bounds__(PT + 32, 1) k_probe_tc(const ProbeArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    // full[s]: centroid stage s loaded; accf[b]: accumulator b written (MMAs
    // done, which also frees the stage they read); acce[b]: accumulator b read
    // by all 8 epilogue warps; aready: the query tile is in shared memory
    __shared__ __align__(8) uint64_t full[2], accf[2], acce[2], aready;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    __shared__ uint64_t wbuf[PT / 32][64];
    // per query of the tile: the smallest n-th-smallest key over its queues;
    // no key at or above it can be among the query's n nearest lists
    __shared__ unsigned long long tau_sh[PQ];
    const int Kp = a.Kp;
    const uint32_t half_bytes = (uint32_t)PN * Kp * 2;  // hi (or lo) of one 128-centroid tile
    __nv_bfloat16 *Ahi = reinterpret_cast<__nv_bfloat16 *>(sm);
    __nv_bfloat16 *Alo = Ahi + PQ * Kp;
    unsigned char *Bs = sm + (size_t)2 * PQ * Kp * 2;  // 2 stages x (hi, lo)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t g0 = (int64_t)blockIdx.x * a.per;
    const int64_t g1 = min(a.total, g0 + a.per);
    if (g0 >= g1) return;
    const int ntiles = (int)(g1 - g0);

    if (warp == 0) tc::tmem_alloc(&tmem_base, 2 * PN);
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&accf[i], 1);
            tc::mbar_init(&acce[i], PT / 32);
        }
        tc::mbar_init(&aready, 1);
        abort_flag = 0;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = tmem_base;

    if (warp == PT / 32) {
        // ---- producer: centroid tiles in, MMAs out (one thread) ----
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16_f32(PQ, PN);
            const uint32_t sbo = (uint32_t)(Kp / 8) * 128u;
            const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo);
            int kl0 = -1, kl1 = -1;  // tile whose copy into stage 0 / 1 is in flight
            int committed = -1;      // last tile whose MMAs were committed
            bool ok = true;
            auto issue_load = [&](int s, int kt) {
                const int t128 = (int)((g0 + kt) % a.nt);
                const __nv_bfloat16 *hi =
                    a.tiles + (size_t)(t128 >> 1) * 2 * 256 * Kp + (size_t)(t128 & 1) * PN * Kp;
                unsigned char *dst = Bs + (size_t)s * 2 * half_bytes;
                tc::mbar_expect_tx(&full[s], 2 * half_bytes);
                tc::bulk_g2s(dst, hi, half_bytes, &full[s]);
                tc::bulk_g2s(dst + half_bytes, hi + (size_t)256 * Kp, half_bytes, &full[s]);
                if (s == 0) kl0 = kt;
                else kl1 = kt;
            };
            issue_load(0, 0);
            if (ntiles > 1) issue_load(1, 1);
            int segi = 0;
            int64_t seg_end = g0;  // first tile past the current query tile
            for (int k = 0; k < ntiles && ok; ++k) {
                const int64_t g = g0 + k;
                if (g >= seg_end) {  // a new query tile: wait until its queries are in place
                    seg_end = (g / a.nt + 1) * a.nt;
                    ok = tc::mbar_wait(&aready, segi & 1, PWAIT);
                    ++segi;
                    if (!ok) break;
                    tc::fence_after();
                }
                const int s = k & 1;
                ok = tc::mbar_wait(&full[s], (k >> 1) & 1, PWAIT);
                if (ok && k >= 2) ok = tc::mbar_wait(&acce[s], ((k - 2) >> 1) & 1, PWAIT);
                if (!ok || abort_flag) break;
                if (s == 0) kl0 = -1;
                else kl1 = -1;
                tc::fence_after();
                const uint32_t bh = tc::smem_u32(Bs + (size_t)s * 2 * half_bytes), bl = bh + half_bytes;
                const uint32_t acc = tbase + (uint32_t)s * PN;
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
                tc::mma_commit(&accf[s]);
                committed = k;
                // the other stage (tile k - 1) takes tile k + 1 once MMA k - 1 is done
                if (k >= 1 && k + 1 < ntiles) {
                    ok = tc::mbar_wait(&accf[s ^ 1], ((k - 1) >> 1) & 1, PWAIT);
                    if (!ok) break;
                    issue_load(s ^ 1, k + 1);
                }
            }
            if (!ok) {
                atomicOr(a.err, DEV_ERR_TIMEOUT);
                abort_flag = 1;
            }
            // nothing may be in flight when shared and tensor memory are released
            if (committed >= 0) tc::mbar_wait(&accf[committed & 1], (committed >> 1) & 1, PWAIT);
            if (kl0 >= 0) tc::mbar_wait(&full[0], (kl0 >> 1) & 1, PWAIT);
            if (kl1 >= 0) tc::mbar_wait(&full[1], (kl1 >> 1) & 1, PWAIT);
        }
    } else {
        // ---- epilogue: 8 warps, two per lane quadrant, one column half each ----
        const int quad = warp & 3, colh = warp >> 2;
        unsigned long long *tsh = tau_sh + quad * 32;
        int segi = 0;
        int k = 0;
        bool failed = false;
        while (k < ntiles && !failed) {
            const int64_t g = g0 + k;
            const int64_t qt = g / a.nt;
            const int nseg = (int)(min(g1, (qt + 1) * a.nt) - g);
            const int seg = (int)(blockIdx.x - (qt * a.nt) / a.per);
            const int64_t r0 = qt * PQ;
            // A: this query tile as bf16 hi/lo (every MMA of the previous tile is done:
            // its last accumulator was read above)
            for (int e = tid; e < PQ * Kp; e += PT) {
                const int r = e / Kp, kk = e - r * Kp;
                const float x = (r0 + r < a.rows && kk < a.d) ? a.q[(r0 + r) * a.d + kk] : 0.f;
                __nv_bfloat16 h, l;
                tc::split_bf16(x, h, l);
                const uint32_t o = tc::core_offset(r, kk, Kp) >> 1;
                Ahi[o] = h;
                Alo[o] = l;
            }
            if (tid < PQ) tau_sh[tid] = KEY_INF;
            tc::fence_proxy_async();
            asm volatile("bar.sync 1, %0;" ::"n"(PT) : "memory");
            if (tid == 0) tc::mbar_arrive(&aready);
            ++segi;
            const int64_t row = r0 + quad * 32 + lane;
            const bool rv = row < a.rows;
            float qn = 0.f;
            if (rv)
                for (int kk = 0; kk < a.d; ++kk) {
                    const float x = a.q[row * a.d + kk];
                    qn = fmaf(x, x, qn);
                }
            uint64_t *myq = rv ? a.lists + (((size_t)row * a.segmax + seg) * 2 + colh) * a.cap : nullptr;
            unsigned long long *gt = rv ? a.gtau + row : nullptr;
            int cnt = 0, nsorted = 0;
            // one 32-column chunk of this thread's row: make room, then append
            // every key below the query's threshold
            auto chunk = [&](float(&v)[32], float cl, int l0) {
                uint32_t need = __ballot_sync(FULL, rv && cnt + 32 > a.cap);
                while (need) {
                    const int src = __ffs(need) - 1;
                    compact<R>(myq, cnt, nsorted, tsh, gt, src, a.n, wbuf[warp]);
                    need &= need - 1;
                }
                const uint64_t tau = *reinterpret_cast<volatile unsigned long long *>(tsh + lane);
                const float tau_d = tau == KEY_INF ? INFINITY : o2f((uint32_t)(tau >> 32));
                const uint32_t vmask =
                    l0 + 32 <= a.nlist ? FULL : (l0 >= a.nlist ? 0u : (1u << (a.nlist - l0)) - 1u);
                uint32_t pass = 0;
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    v[e] = qn - 2.f * v[e] + __shfl_sync(FULL, cl, e);
                    pass |= (v[e] <= tau_d ? 1u : 0u) << e;
                }
                pass &= rv ? vmask : 0u;
                if (pass) {
#pragma unroll
                    for (int e = 0; e < 32; ++e)
                        if ((pass >> e) & 1u) {
                            const uint64_t key = make_key(v[e], (uint32_t)(l0 + e));
                            if (key < tau) myq[cnt++] = key;
                        }
                }
            };
            for (int i = 0; i < nseg; ++i, ++k) {
                const int b = k & 1;
                const int lbase = (int)((g0 + k) % a.nt) * PN + colh * 64;
                // |c|^2 of this lane's column in each 32-column chunk, and the
                // query's threshold from the other CTAs on its query tile
                const float cl0 = lbase + lane < a.nlist ? __ldg(a.cnorm + lbase + lane) : 0.f;
                const float cl1 = lbase + 32 + lane < a.nlist ? __ldg(a.cnorm + lbase + 32 + lane) : 0.f;
                const unsigned long long gtv = (rv && colh == 0) ? *(volatile unsigned long long *)gt : KEY_INF;
                bool ok = tc::mbar_wait(&accf[b], (k >> 1) & 1, PWAIT);
                ok = __all_sync(FULL, ok) && !abort_flag;
                if (!ok) {
                    failed = true;
                    break;
                }
                tc::fence_after();
                float v0[32], v1[32];
                const uint32_t taddr = tbase + ((uint32_t)(quad * 32) << 16) + (uint32_t)b * PN + colh * 64;
                tc::tmem_ld32(taddr, v0);
                tc::tmem_ld32(taddr + 32, v1);
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&acce[b]);
                if (gtv != KEY_INF) atomicMin(tsh + lane, gtv);
                chunk(v0, cl0, lbase);
                chunk(v1, cl1, lbase + 32);
            }
            if (failed) {
                abort_flag = 1;
                if (lane == 0) atomicOr(a.err, DEV_ERR_TIMEOUT);
            } else {
                // every queue of this range down to its sorted n smallest
                uint32_t m = __ballot_sync(FULL, rv);
                while (m) {
                    const int src = __ffs(m) - 1;
                    compact<R>(myq, cnt, nsorted, tsh, gt, src, a.n, wbuf[warp]);
                    m &= m - 1;
                }
            }
            // the thresholds and the queries are replaced only after every epilogue
            // warp is done; a failure anywhere ends every epilogue warp here
            asm volatile("bar.sync 1, %0;" ::"n"(PT) : "memory");
            failed = abort_flag != 0;
        }
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
    p.bytes = (size_t)nq * p.segmax * 2 * p.cap * sizeof(uint64_t) + (size_t)nq * sizeof(uint64_t);
    return p;
}

template <int R>
void launch_r(const ProbeArgs &a, const ProbePlan &p, int smem, int32_t *probes, int32_t stride,
              cudaStream_t st) {
    FA_CHECK_CUDA(cudaFuncSetAttribute(k_probe_tc<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_probe_tc<R><<<p.grid, PT + 32, smem, st>>>(a);
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
    a.gtau = reinterpret_cast<unsigned long long *>(scratch + (size_t)nq * p.segmax * 2 * p.cap);
    a.err = err;
    FA_CHECK_CUDA(cudaMemsetAsync(a.gtau, 0xFF, sizeof(uint64_t) * nq, st));
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
