// Coarse probe (step 2) on the tensor cores, as two kernels:
//
//   k_coarse_dist_tc   d2(q, c_l) = |q|^2 - 2 q.c_l + |c_l|^2 for a block of
//                      queries and every centroid, into a distance block in HBM;
//   k_select_rows      each query's nprobe nearest lists from its row.
//
// Distances: queries and centroids are split into bf16 pairs hi + lo
// (x ~= hi + lo to about 16 significant bits); each K-step takes three MMAs
// (hi.hi + hi.lo + lo.hi) with FP32 accumulation in tensor memory, close to
// FP32 accuracy at bf16 tensor rate. The (query tile, centroid tile) pairs of
// the block are laid out query-tile major and cut into one contiguous range
// per CTA, so every SM gets the same number of MMA tiles; a CTA whose range
// crosses into the next query tile reloads its queries there.
//
// The MMA takes the centroid tile as its M side and the query tile as its N
// side, so tensor-memory lane i holds centroid i's dot products with the 128
// queries: for each query the 32 lanes of a warp then store 32 consecutive
// distances of that query's row, one full 128-byte line per store.
// The CTA is warp-specialized:
//   - one producer thread streams 128-centroid tiles into a two-stage shared-
//     memory ring with bulk copies and issues the MMAs of each tile into one
//     of two tensor-memory accumulators; mbarriers order the copies, the MMAs
//     and the epilogue, so the MMAs of tile i run while tile i-1 is written;
//   - 8 epilogue warps, two per tensor-memory lane quadrant (32 centroids)
//     and one half of the queries each, read an accumulator into registers,
//     hand it back at once, and store their 32 centroids x 64 queries.
//
// Selection reads each row once with several 16-byte loads in flight per lane
// and keeps the row's n smallest keys (distance, list id) in the warp's
// registers (warp_topk.cuh): the result is the sorted top-n, ties by list id.
#include <algorithm>
#include <vector>

#include "../fa_internal.h"
#include "tc_util.cuh"
#include "warp_topk.cuh"

namespace fa {

namespace {

constexpr int PQ = 128;  // queries per tile (MMA N)
constexpr int PN = 128;  // centroids per tile (MMA M = tensor-memory lanes)
constexpr int PT = 256;  // epilogue threads: 8 warps
constexpr uint32_t PWAIT = 1u << 22;

// Centroid tiles are cut along K into KC contiguous chunks (two when the
// padded dimension allows chunks of whole 16-wide K-steps), so that the
// shared-memory ring of two tiles holds 2 KC chunks and a chunk is refilled
// as soon as its own MMAs are done.
__host__ __device__ constexpr int kchunks(int Kp) { return Kp % 32 == 0 ? 2 : 1; }

struct DistArgs {
    const float *q;              // [rows][d] the block's queries
    int64_t rows;
    int32_t d, Kp;
    const __nv_bfloat16 *tiles;  // [nt][KC][hi, lo][PN * Kp / KC], core-matrix layout
    const float *cnorm;          // [nlist] |c|^2
    int32_t nlist, nt;
    int64_t total;               // query tiles * nt
    int32_t per;                 // (query tile, centroid tile) pairs per CTA
    float *D;                    // [rows][ldd], ldd a multiple of 4
    int64_t ldd;
    uint32_t *err;
    int32_t ip;                  // the negated inner product -q.c instead of the squared L2
};

__global__ void __launch_bounds__(PT + 32, 1) k_coarse_dist_tc(const DistArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    // full[s] / sfree[s]: centroid chunk stage s loaded / read by its MMAs;
    // accf[b]: accumulator b written; acce[b]: accumulator b read by all 8
    // epilogue warps; aready: the query tile is in place
    __shared__ __align__(8) uint64_t full[4], sfree[4], accf[2], acce[2], aready;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    __shared__ float qn_sh[PQ];  // |q|^2 of the current query tile
    const int Kp = a.Kp;
    const int KC = kchunks(Kp), Kc = Kp / KC, S = 2 * KC;
    const uint32_t chunk_bytes = (uint32_t)2 * PN * Kc * 2;  // hi + lo of one K-chunk
    __nv_bfloat16 *Ahi = reinterpret_cast<__nv_bfloat16 *>(sm);
    __nv_bfloat16 *Alo = Ahi + PQ * Kp;
    unsigned char *Bs = sm + (size_t)2 * PQ * Kp * 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t g0 = (int64_t)blockIdx.x * a.per;
    const int64_t g1 = min(a.total, g0 + a.per);
    if (g0 >= g1) return;
    const int ntiles = (int)(g1 - g0);

    if (warp == 0) tc::tmem_alloc(&tmem_base, 2 * PN);
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&sfree[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
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
        // ---- producer: centroid chunks in, MMAs out (one thread) ----
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16_f32(PN, PQ);
            const uint32_t sbo_q = (uint32_t)(Kp / 8) * 128u, sbo_c = (uint32_t)(Kc / 8) * 128u;
            const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo);
            const int nch = ntiles * KC;
            int issued = 0, consumed = 0;  // chunks copied in / read by MMAs (in order)
            int committed = -1;            // last tile whose MMAs were committed
            bool ok = true;
            auto issue_load = [&](int c) {
                const int t = (int)((g0 + c / KC) % a.nt);
                const int st = c % S;
                tc::mbar_expect_tx(&full[st], chunk_bytes);
                tc::bulk_g2s(Bs + (size_t)st * chunk_bytes,
                             a.tiles + ((size_t)t * KC + c % KC) * 2 * PN * Kc, chunk_bytes, &full[st]);
                ++issued;
            };
            while (issued < min(S, nch)) issue_load(issued);
            int segi = 0;
            int64_t seg_end = g0;  // first pair past the current query tile
            for (int c = 0; c < nch; ++c) {
                const int k = c / KC, h = c % KC, st = c % S, b = k & 1;
                if (h == 0) {
                    const int64_t g = g0 + k;
                    if (g >= seg_end) {  // a new query tile: wait until its queries are in place
                        seg_end = (g / a.nt + 1) * a.nt;
                        ok = tc::mbar_wait(&aready, segi & 1, PWAIT);
                        ++segi;
                        if (!ok) break;
                    }
                    // accumulator b is free once the epilogue has read tile k - 2
                    if (k >= 2) ok = tc::mbar_wait(&acce[b], ((k - 2) >> 1) & 1, PWAIT);
                }
                if (ok) ok = tc::mbar_wait(&full[st], (c / S) & 1, PWAIT);
                if (!ok || abort_flag) break;
                ++consumed;
                tc::fence_after();
                const uint32_t ch = tc::smem_u32(Bs + (size_t)st * chunk_bytes), cl = ch + chunk_bytes / 2;
                const uint32_t acc = tbase + (uint32_t)b * PN;
                for (int kk = 0; kk < Kc / 16; ++kk) {
                    const int ks = h * (Kc / 16) + kk;  // K-step within the tile
                    const uint64_t dch = tc::smem_desc(ch + 256u * kk, 128, sbo_c);
                    const uint64_t dcl = tc::smem_desc(cl + 256u * kk, 128, sbo_c);
                    const uint64_t dqh = tc::smem_desc(ah + 256u * ks, 128, sbo_q);
                    const uint64_t dql = tc::smem_desc(al + 256u * ks, 128, sbo_q);
                    // centroids (stage) as A, queries as B
                    tc::mma_bf16(acc, dch, dqh, idesc, ks > 0 ? 1u : 0u);
                    tc::mma_bf16(acc, dch, dql, idesc, 1u);
                    tc::mma_bf16(acc, dcl, dqh, idesc, 1u);
                }
                tc::mma_commit(&sfree[st]);
                if (h == KC - 1) {
                    tc::mma_commit(&accf[b]);
                    committed = k;
                }
                // the stage of chunk c - 1 takes chunk c - 1 + S once its MMAs are done
                if (c >= 1 && issued < nch) {
                    ok = tc::mbar_wait(&sfree[(c - 1) % S], ((c - 1) / S) & 1, PWAIT);
                    if (!ok) break;
                    issue_load(issued);
                }
            }
            if (!ok) {
                atomicOr(a.err, DEV_ERR_TIMEOUT);
                abort_flag = 1;
            }
            // nothing may be in flight when shared and tensor memory are released
            if (committed >= 0) tc::mbar_wait(&accf[committed & 1], (committed >> 1) & 1, PWAIT);
            for (int c = consumed; c < issued; ++c) tc::mbar_wait(&full[c % S], (c / S) & 1, PWAIT);
        }
    } else {
        // ---- epilogue: 8 warps; lane quadrant = 32 centroids, half = 64 queries ----
        const int quad = warp & 3, colh = warp >> 2;
        int k = 0;
        bool failed = false;
        while (k < ntiles && !failed) {
            const int64_t qt = (g0 + k) / a.nt;
            const int nseg = (int)(min(g1, (qt + 1) * a.nt) - (g0 + k));
            const int64_t r0 = qt * PQ;
            // this query tile as bf16 hi/lo, and |q|^2; every MMA on the
            // previous one is done (its last accumulator was read below)
            for (int e = tid; e < PQ * Kp; e += PT) {
                const int r = e / Kp, kk = e - r * Kp;
                const float x = (r0 + r < a.rows && kk < a.d) ? a.q[(r0 + r) * a.d + kk] : 0.f;
                __nv_bfloat16 h, l;
                tc::split_bf16(x, h, l);
                const uint32_t o = tc::core_offset(r, kk, Kp) >> 1;
                Ahi[o] = h;
                Alo[o] = l;
            }
            if (tid < PQ) {
                float qn = 0.f;
                if (r0 + tid < a.rows)
                    for (int kk = 0; kk < a.d; ++kk) {
                        const float x = a.q[(r0 + tid) * a.d + kk];
                        qn = fmaf(x, x, qn);
                    }
                qn_sh[tid] = qn;
            }
            tc::fence_proxy_async();
            asm volatile("bar.sync 1, %0;" ::"n"(PT) : "memory");
            if (tid == 0) tc::mbar_arrive(&aready);
            // |q|^2 of query colh * 64 + 32 c + lane, for the broadcasts below
            const float qn0 = qn_sh[colh * 64 + lane], qn1 = qn_sh[colh * 64 + 32 + lane];
            const int64_t rq = r0 + colh * 64;  // first query of this warp's half
            // 32 queries (j0 + e) x this lane's centroid l: row j0 + e, column l
            auto store_chunk = [&](const float(&v)[32], float qnl, int j0, int l, float cn) {
                const int64_t first = rq + j0;
                const int64_t left = a.rows - first;
                const int nrow = left <= 0 ? 0 : (left >= 32 ? 32 : (int)left);
                float *p = a.D + first * a.ldd + l;
                const bool lv = l < a.nlist;
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    const float dd = a.ip ? -v[e] : __shfl_sync(FULL, qnl, e) - 2.f * v[e] + cn;
                    if (lv && e < nrow) *p = dd;
                    p += a.ldd;
                }
            };
            for (int i = 0; i < nseg; ++i, ++k) {
                const int b = k & 1;
                const int l = (int)((g0 + k) % a.nt) * PN + quad * 32 + lane;
                const float cn = l < a.nlist ? __ldg(a.cnorm + l) : 0.f;
                bool ok = tc::mbar_wait(&accf[b], (k >> 1) & 1, PWAIT);
                ok = __all_sync(FULL, ok) && !abort_flag;
                if (!ok) {
                    failed = true;
                    break;
                }
                tc::fence_after();
                // read, store, read the next 32 columns: the accumulator goes
                // back after both, well within the next tile's MMA time
                const uint32_t taddr = tbase + ((uint32_t)(quad * 32) << 16) + (uint32_t)b * PN + colh * 64;
                float v[32];
                tc::tmem_ld32(taddr, v);
                store_chunk(v, qn0, 0, l, cn);
                tc::tmem_ld32(taddr + 32, v);
                store_chunk(v, qn1, 32, l, cn);
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&acce[b]);
            }
            if (failed) {
                abort_flag = 1;
                if (lane == 0) atomicOr(a.err, DEV_ERR_TIMEOUT);
            }
            // the queries are replaced only after every epilogue warp is done;
            // a failure anywhere ends every epilogue warp here
            asm volatile("bar.sync 1, %0;" ::"n"(PT) : "memory");
            failed = abort_flag != 0;
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_free(tbase, 2 * PN);
}

// One warp per row: the n smallest (distance, column) keys of D[row][0, nc).
// Rows are 16-byte aligned (ldd a multiple of 4); each lane keeps U 16-byte
// loads of the next batch in flight while it offers the current one. The
// kernel is issue-bound on its pushes and merges, so three CTAs per SM (80
// registers, no spills at n <= 256) beat two (0.59 -> ~0.5 ms per 10k rows of
// 16384).
template <int R>
__global__ void __launch_bounds__(256, 3) k_select_rows(const float *__restrict__ D, int64_t ldd, int64_t nrows,
                                                     int32_t nc, int32_t ntop, int32_t *__restrict__ out_ids,
                                                     int32_t out_stride) {
    constexpr int U = 4;
    __shared__ uint64_t wbuf[8][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * 8 + warp;
    if (row >= nrows) return;
    WarpTopK<R> tk;
    tk.init(wbuf[warp], ntop);
    const float4 *d4 = reinterpret_cast<const float4 *>(D + row * ldd);
    const int n4 = (nc + 3) >> 2;
    float4 cur[U], nxt[U];
    float thr_f = INFINITY;  // the distance of the n-th smallest key so far
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int i = lane + 32 * u;
        cur[u] = i < n4 ? __ldg(d4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int base = 0; base < n4; base += 32 * U) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = base + 32 * U + lane + 32 * u;
            nxt[u] = i < n4 ? __ldg(d4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // most keys lose to the n-th smallest so far: one float test per 16
        // bytes, and a single (not unrolled) push site for the rest, so the
        // bitonic merges appear once in the code
        uint32_t todo = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = 4 * (base + lane + 32 * u);
            const float mn = fminf(fminf(cur[u].x, cur[u].y), fminf(cur[u].z, cur[u].w));
            todo |= (__any_sync(FULL, c < nc && mn <= thr_f) ? 1u : 0u) << u;
        }
#pragma unroll 1
        for (; todo; todo &= todo - 1) {
            const int u = __ffs(todo) - 1;
            const float4 x = u == 0 ? cur[0] : u == 1 ? cur[1] : u == 2 ? cur[2] : cur[3];
            const int c = 4 * (base + lane + 32 * u);
#pragma unroll 1
            for (int j = 0; j < 4; ++j) {
                const float v = j == 0 ? x.x : j == 1 ? x.y : j == 2 ? x.z : x.w;
                tk.push(make_key(v, (uint32_t)(c + j)), c + j < nc);
            }
            thr_f = tk.thr == KEY_INF ? INFINITY : o2f((uint32_t)(tk.thr >> 32));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) cur[u] = nxt[u];
    }
    tk.finish();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = r * 32 + lane;
        if (e < ntop) {
            const uint64_t k = tk.L[r];
            out_ids[row * out_stride + e] = k == KEY_INF ? -1 : (int32_t)(k & 0xffffffffu);
        }
    }
}

template <int R>
void select_r(const float *D, int64_t ldd, int64_t rows, int32_t nc, int32_t ntop, int32_t *out,
              int32_t stride, cudaStream_t st) {
    k_select_rows<R><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(D, ldd, rows, nc, ntop, out, stride);
    FA_CHECK_CUDA(cudaGetLastError());
}

}  // namespace

// Centroids as tensor-core tiles: [nt][KC][hi, lo][PN rows x Kp / KC] in
// core-matrix layout (each K-chunk contiguous), rows past nlist zero.
// Host-side preparation at index upload.
void prepare_centroid_tiles(const float *cent, int32_t nlist, int32_t d, std::vector<uint16_t> &out,
                            int32_t &Kp, int32_t &ntiles) {
    Kp = (d + 15) / 16 * 16;
    ntiles = (nlist + PN - 1) / PN;
    const int KC = kchunks(Kp), Kc = Kp / KC;
    out.assign((size_t)ntiles * 2 * PN * Kp, 0);
    for (int l = 0; l < nlist; ++l) {
        const int t = l / PN, r = l % PN;
        for (int k = 0; k < d; ++k) {
            const int h = k / Kc, kc = k % Kc;
            uint16_t *hi = out.data() + ((size_t)t * KC + h) * 2 * PN * Kc;
            uint16_t *lo = hi + (size_t)PN * Kc;
            const float x = cent[(size_t)l * d + k];
            const uint16_t hb = tc::host_bf16_bits(x);
            const uint32_t o = tc::core_offset(r, kc, Kc) >> 1;
            hi[o] = hb;
            lo[o] = tc::host_bf16_bits(x - tc::host_bf16_float(hb));
        }
    }
}

int64_t coarse_tc_ldd(int32_t nlist) { return ((int64_t)nlist + 3) & ~3ll; }

void launch_coarse_tc(const DeviceIndex &ix, const float *q, int64_t rows, int32_t ntop, float *D,
                      int32_t *probes, int32_t probe_stride, uint32_t *err, cudaStream_t st) {
    if (rows == 0) return;
    FA_REQUIRE(ix.centroids_bf16 != nullptr, FA_ERR_ARG, "tensor-core centroid tiles missing");
    FA_REQUIRE(ntop >= 1 && ntop <= 512, FA_ERR_ARG, "top-n of the coarse probe must be in 1..512");
    DistArgs a{};
    a.q = q;
    a.rows = rows;
    a.d = ix.d;
    a.Kp = ix.tc_kp;
    a.tiles = reinterpret_cast<const __nv_bfloat16 *>(ix.centroids_bf16);
    a.cnorm = ix.cnorm;
    a.ip = ix.metric == FA_METRIC_IP ? 1 : 0;
    a.nlist = ix.nlist;
    a.nt = ix.tc_ntiles;
    a.total = (rows + PQ - 1) / PQ * (int64_t)a.nt;
    a.per = (int32_t)((a.total + cur_num_sms() - 1) / cur_num_sms());
    a.D = D;
    a.ldd = coarse_tc_ldd(ix.nlist);
    a.err = err;
    const int grid = (int)((a.total + a.per - 1) / a.per);
    // queries + two centroid stages; at least 116 KB so that one CTA (256
    // tensor-memory columns) runs per SM and allocation never waits
    FA_REQUIRE(a.Kp <= 128, FA_ERR_ARG, "tensor-core coarse probe supports d <= 128");
    const int smem = std::max(3 * 2 * PQ * a.Kp * 2, 116 * 1024);
    FA_CHECK_CUDA(cudaFuncSetAttribute(k_coarse_dist_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_coarse_dist_tc<<<grid, PT + 32, smem, st>>>(a);
    FA_CHECK_CUDA(cudaGetLastError());
    const int64_t ldd = a.ldd;
    if (ntop <= 32) select_r<1>(D, ldd, rows, ix.nlist, ntop, probes, probe_stride, st);
    else if (ntop <= 64) select_r<2>(D, ldd, rows, ix.nlist, ntop, probes, probe_stride, st);
    else if (ntop <= 128) select_r<4>(D, ldd, rows, ix.nlist, ntop, probes, probe_stride, st);
    else if (ntop <= 256) select_r<8>(D, ldd, rows, ix.nlist, ntop, probes, probe_stride, st);
    else select_r<16>(D, ldd, rows, ix.nlist, ntop, probes, probe_stride, st);
}

}  // namespace fa
