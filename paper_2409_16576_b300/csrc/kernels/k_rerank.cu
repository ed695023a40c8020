// Output stage of the filtering path and the heuristic re-rank (step 8).
//
// k_finish   the ADC top-k of each query mapped to the caller's ids and
//            ordered by (distance, caller id)
// k_rerank   Algorithm 1 (§4.2): the ADC top-n candidates, in ascending ADC
//            order, are re-ranked in mini-batches of BatchSize on exact
//            squared L2 distances over the raw vectors. Q (the max-heap of
//            the paper) holds the k smallest (distance, id) pairs seen; after
//            each mini-batch the change rate of Eq. 3,
//               Delta = |S_n - S_n intersect S_{n-1}| / k,
//            is compared with eps: Delta <= eps increments a stability
//            counter, otherwise it is reset, and the loop ends when the
//            counter reaches beta.
// One warp handles one query. Eight lanes read a candidate's raw row in
// consecutive 16-byte pieces (a full 128-byte request for d = 128 uint8), so
// rows in pinned host memory cross the host link in full-line reads; the 32
// rows of a mini-batch step are issued back to back before any is summed.
#include "../fa_internal.h"
#include "rerank_rows.cuh"
#include "warp_topk.cuh"

namespace fa {

template <int R>
__global__ void __launch_bounds__(256) k_finish(const uint64_t *__restrict__ topkeys, int64_t nq,
                                                int32_t ntop, int32_t k, const int32_t *kq,
                                                const int64_t *__restrict__ perm,
                                                int64_t *__restrict__ out_ids,
                                                float *__restrict__ out_dist) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t qi = (int64_t)blockIdx.x * 8 + warp;
    if (qi >= nq) return;
    int kk = kq ? kq[qi] : k;
    kk = kk < 1 ? 1 : (kk > k ? k : kk);
    uint64_t L[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = r * 32 + lane;
        uint64_t key = KEY_INF;
        if (e < kk && e < ntop) key = topkeys[qi * ntop + e];
        if (key != KEY_INF) {
            const uint32_t internal = (uint32_t)(key & 0xffffffffu);
            key = (key & 0xffffffff00000000ull) | (uint32_t)perm[internal];
        }
        L[r] = key;
    }
    bitonic_sort<R>(L);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = r * 32 + lane;
        if (e < k) {
            const uint64_t key = (e < kk) ? L[r] : KEY_INF;
            out_ids[qi * k + e] = key == KEY_INF ? -1 : (int64_t)(key & 0xffffffffu);
            out_dist[qi * k + e] = key == KEY_INF ? INFINITY : o2f((uint32_t)(key >> 32));
        }
    }
}

// k > 256: one CTA per query sorts the row by (distance, caller id) in shared memory.
__global__ void __launch_bounds__(512) k_finish_big(const uint64_t *__restrict__ topkeys, int64_t nq,
                                                    int32_t ntop, int32_t k, const int32_t *kq,
                                                    const int64_t *__restrict__ perm, int KP,
                                                    int64_t *__restrict__ out_ids,
                                                    float *__restrict__ out_dist) {
    extern __shared__ uint64_t keys[];
    const int64_t qi = blockIdx.x;
    int kk = kq ? kq[qi] : k;
    kk = kk < 1 ? 1 : (kk > k ? k : kk);
    for (int e = threadIdx.x; e < KP; e += blockDim.x) {
        uint64_t key = KEY_INF;
        if (e < kk && e < ntop) key = topkeys[qi * ntop + e];
        if (key != KEY_INF) {
            const uint32_t internal = (uint32_t)(key & 0xffffffffu);
            key = (key & 0xffffffff00000000ull) | (uint32_t)perm[internal];
        }
        keys[e] = key;
    }
    __syncthreads();
    for (int size = 2; size <= KP; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < KP / 2; i += blockDim.x) {
                const int lo = ((i & ~(stride - 1)) << 1) | (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const uint64_t p = keys[lo], q = keys[hi];
                if ((p > q) == up) {
                    keys[lo] = q;
                    keys[hi] = p;
                }
            }
            __syncthreads();
        }
    for (int e = threadIdx.x; e < k; e += blockDim.x) {
        const uint64_t key = e < kk ? keys[e] : KEY_INF;
        out_ids[qi * k + e] = key == KEY_INF ? -1 : (int64_t)(key & 0xffffffffu);
        out_dist[qi * k + e] = key == KEY_INF ? INFINITY : o2f((uint32_t)(key >> 32));
    }
}

void launch_finish(const DeviceIndex &ix, const uint64_t *topkeys, int64_t nq, int32_t ntop,
                   int32_t k, const int32_t *kq, int64_t *out_ids, float *out_dist,
                   cudaStream_t st) {
    if (nq == 0) return;
    if (k > 256) {
        FA_REQUIRE(k <= 16384, FA_ERR_ARG, "k above 16384");
        int KP = 1;
        while (KP < k) KP <<= 1;
        FA_CHECK_CUDA(cudaFuncSetAttribute(k_finish_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           KP * 8));
        k_finish_big<<<(unsigned)nq, 512, KP * 8, st>>>(topkeys, nq, ntop, k, kq, ix.perm, KP,
                                                          out_ids, out_dist);
        FA_CHECK_CUDA(cudaGetLastError());
        return;
    }
    const dim3 grid((unsigned)((nq + 7) / 8));
    if (k <= 32)
        k_finish<1><<<grid, 256, 0, st>>>(topkeys, nq, ntop, k, kq, ix.perm, out_ids, out_dist);
    else if (k <= 64)
        k_finish<2><<<grid, 256, 0, st>>>(topkeys, nq, ntop, k, kq, ix.perm, out_ids, out_dist);
    else if (k <= 128)
        k_finish<4><<<grid, 256, 0, st>>>(topkeys, nq, ntop, k, kq, ix.perm, out_ids, out_dist);
    else
        k_finish<8><<<grid, 256, 0, st>>>(topkeys, nq, ntop, k, kq, ix.perm, out_ids, out_dist);
    FA_CHECK_CUDA(cudaGetLastError());
}

// Page buffer of one warp for the paged re-rank (§4.3): pages read so far by
// the warp's current query, found through an open-addressing table whose
// entries carry the query's generation (so no table clearing per query).
struct PagedCtx {
    const uint32_t *vpage;  // [n] page of each caller id
    const uint16_t *vslot;  // [n] row of each caller id in its page
    const uint8_t *pages;   // the pages (mapped pinned host memory), page_bytes apart
    uint8_t *cache;         // this warp's buffer: cap_pages pages
    uint64_t *table;        // [tsize] (generation << 32) | (page + 1), 0 = empty
    uint32_t *tslot;        // [tsize] buffer slot of each entry
    int32_t tsize, page_rows, page_bytes;
    uint32_t gen;           // generation of the current query
    int32_t nread;          // pages the current query read
};

// Rows of the 32 tasks of a step (uid = caller id, < 0 = none) resolved to
// rows of the warp's page buffer: the distinct pages of the step are looked
// up once each (one lane per page), the ones not yet buffered are copied
// from the slow tier by the whole warp, 16 bytes a lane. Warp-collective.
__device__ __forceinline__ int64_t paged_row(PagedCtx &pg, int64_t uid) {
    const int lane = threadIdx.x & 31;
    const bool need = uid >= 0;
    const uint32_t p = need ? pg.vpage[uid] : 0xffffffffu;
    const uint32_t peers = __match_any_sync(FULL, p);
    const int leader = __ffs(peers) - 1;
    const bool lead = need && lane == leader;
    const uint64_t key = ((uint64_t)pg.gen << 32) | (uint64_t)(p + 1u);
    const uint32_t tmask = (uint32_t)(pg.tsize - 1);
    const uint32_t h0 = (p * 2654435761u) & tmask;
    int32_t slot = -1;
    if (lead) {  // lookups in parallel (the table holds at most half its size)
        uint32_t h = h0;
        for (int probe = 0; probe < pg.tsize; ++probe) {
            const uint64_t e = pg.table[h];
            if (e == key) {
                slot = (int32_t)pg.tslot[h];
                break;
            }
            if ((uint32_t)(e >> 32) != pg.gen) break;  // empty for this query: p is new
            h = (h + 1) & tmask;
        }
    }
    const uint32_t miss = __ballot_sync(FULL, lead && slot < 0);
    if (lead && slot < 0) slot = pg.nread + __popc(miss & ((1u << lane) - 1u));
    // insertions one lane at a time: two new pages may probe the same entry
    for (uint32_t mm = miss; mm; mm &= mm - 1) {
        if (lane == __ffs(mm) - 1) {
            uint32_t h = h0;
            for (int probe = 0; probe < pg.tsize; ++probe) {
                if ((uint32_t)(pg.table[h] >> 32) != pg.gen) break;
                h = (h + 1) & tmask;
            }
            pg.table[h] = key;
            pg.tslot[h] = (uint32_t)slot;
        }
        __syncwarp();
    }
    for (uint32_t mm = miss; mm; mm &= mm - 1) {
        const int src = __ffs(mm) - 1;
        const uint32_t pp = __shfl_sync(FULL, p, src);
        const int32_t ss = __shfl_sync(FULL, slot, src);
        const uint4 *from = reinterpret_cast<const uint4 *>(pg.pages + (size_t)pp * pg.page_bytes);
        uint4 *to = reinterpret_cast<uint4 *>(pg.cache + (size_t)ss * pg.page_bytes);
        for (int o = lane; o < pg.page_bytes / 16; o += 32) to[o] = from[o];
    }
    pg.nread += __popc(miss);
    __syncwarp();
    slot = __shfl_sync(FULL, slot, leader);
    return need ? (int64_t)slot * pg.page_rows + pg.vslot[uid] : (int64_t)-1;
}

template <int R, typename T>
__device__ __forceinline__ void rerank_one(
    const float *__restrict__ q, int32_t d, const uint64_t *__restrict__ topkeys, int64_t qi,
    int32_t ntop, int32_t k, const int32_t *kq, int32_t batch, int32_t beta, float eps,
    const int64_t *__restrict__ perm, const T *__restrict__ raw, int raw_internal,
    int64_t *__restrict__ out_ids, float *__restrict__ out_dist, int32_t *stats, float *qs, int ip,
    PagedCtx *pg = nullptr) {
    const int lane = threadIdx.x & 31;
    __syncwarp();  // the previous query of this warp is done with qs
    for (int j = lane; j < d; j += 32) qs[j] = q[qi * d + j];
    __syncwarp();
    // uint8 rows: an integral query with coordinates in 0..255 takes the
    // integer form (its bytes packed after the floats in qs)
    bool qint = false;
    uint32_t *qp = reinterpret_cast<uint32_t *>(qs + d);
    if (!ip && std::is_same<T, uint8_t>::value && d <= 258 && d % 16 == 0) qint = pack_u8_query(qs, d, qp);
    int kk = kq ? kq[qi] : k;
    kk = kk < 1 ? 1 : (kk > k ? k : kk);
    const uint64_t *tk = topkeys + qi * ntop;
    // tasks: ADC top-n in ascending order; count the valid ones
    int valid = 0;
    for (int e0 = 0; e0 < ntop; e0 += 32) {
        const int e = e0 + lane;
        const bool ok = e < ntop && tk[e] != KEY_INF;
        valid += __popc(__ballot_sync(FULL, ok));
    }
    // row of task e: its internal id when the rows are in internal order,
    // else its caller id (tasks are internal ids)
    auto task_id = [&](int e, int lim) -> int64_t {
        if (e >= lim) return (int64_t)-1;
        const uint32_t v = (uint32_t)(tk[e] & 0xffffffffu);
        return raw_internal ? (int64_t)v : perm[v];
    };
    uint64_t Q[R];
#pragma unroll
    for (int r = 0; r < R; ++r) Q[r] = KEY_INF;
    int counter = 0, batches = 0;
    // the first step's ids; each step fetches the next one's before its rows
    int64_t uid = task_id(lane, batch < valid ? batch : valid);
    for (int i = 0; i < valid; i += batch) {
        uint64_t old[R];
#pragma unroll
        for (int r = 0; r < R; ++r) old[r] = Q[r];
        const int end = i + batch < valid ? i + batch : valid;
        for (int s = i; s < end; s += 32) {
            // next step: the rest of this mini-batch, else the next mini-batch
            int ns = s + 32, nend = end;
            if (ns >= end) {
                ns = end;
                nend = end + batch < valid ? end + batch : valid;
            }
            const int64_t uid_next = task_id(ns + lane, nend);
            if (!pg && uid_next >= 0) {  // the next step's row into L2 while this step's rows load
                const char *rn = reinterpret_cast<const char *>(raw + uid_next * (int64_t)d);
                for (int o = 0; o < d * (int)sizeof(T); o += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(rn + o));
            }
            const float dist = pg ? exact_rows_any<T, true>(reinterpret_cast<const T *>(pg->cache), d, qs, qp,
                                                            qint, paged_row(*pg, uid), ip != 0)
                                  : exact_rows_any<T>(raw, d, qs, qp, qint, uid, ip != 0);
            // only keys below Q's kk-th can change Q's first kk entries (the
            // output and Eq. 3); a step with none leaves them as they are.
            // Keys carry caller ids (ties break by them, as in the oracle):
            // with rows in internal order the id is looked up only when the
            // distance alone does not already rule the key out
            const uint64_t kth = warp_elem<R>(Q, kk - 1);
            int64_t cid = uid;
            if (raw_internal && uid >= 0 && f2o(dist) <= (uint32_t)(kth >> 32)) cid = perm[uid];
            uint64_t key[1] = {uid >= 0 ? make_key(dist, (uint32_t)cid) : KEY_INF};
            if (raw_internal && uid >= 0 && f2o(dist) > (uint32_t)(kth >> 32)) key[0] = KEY_INF;
            const uint32_t in = __ballot_sync(FULL, key[0] < kth);
            if (R == 1 && in && __popc(in) <= 8) {  // few new keys: insert them one at a time
                insert_sorted32(Q[0], key[0], in);
            } else if (in) {
                bitonic_sort<1>(key);
                merge_sorted32<R>(Q, key[0]);
            }
            uid = uid_next;
        }
        ++batches;
        if (eps < 0.f) continue;  // Delta <= eps never holds: no early stop
        // Eq. 3: members of the new top-k that were not in the previous one.
        // Q is the kk smallest of (old Q and the mini-batch), so an old
        // member stays iff it is not above the new kk-th key; the change is
        // the new member count less the members that stayed.
        const uint64_t newmax = warp_elem<R>(Q, kk - 1);
        int now = 0, stayed = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = r * 32 + lane;
            now += __popc(__ballot_sync(FULL, e < kk && Q[r] != KEY_INF));
            stayed += __popc(__ballot_sync(FULL, e < kk && old[r] != KEY_INF && old[r] <= newmax));
        }
        const int changed = now - stayed;
        // Algorithm 1's test on Eq. 3, with this query's own k
        if ((double)changed / (double)kk <= (double)eps) {
            ++counter;
            if (counter >= beta) break;
        } else {
            counter = 0;
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = r * 32 + lane;
        if (e < k) {
            const uint64_t key = e < kk ? Q[r] : KEY_INF;
            out_ids[qi * k + e] = key == KEY_INF ? -1 : (int64_t)(key & 0xffffffffu);
            out_dist[qi * k + e] = key == KEY_INF ? INFINITY : o2f((uint32_t)(key >> 32));
        }
    }
    if (stats && lane == 0) {
        stats[qi * 4 + 2] = batches;
        stats[qi * 4 + 3] = valid;
    }
}

// One warp per query. ctr == null: warp w of CTA b takes query b * warps + w.
// Otherwise the warps are persistent and pull queries from *ctr (zeroed by
// the caller), so a small grid can run beside another kernel without taking
// more than its own warps' share of an SM.
// LEAN: the persistent form run beside a scan; capped at 64 registers so
// that two of its warps fit in what three scan CTAs leave of an SM.
template <int R, typename T, bool LEAN>
__global__ void __launch_bounds__(LEAN ? 32 : 256, LEAN ? 32 : 3) k_rerank(
    const float *__restrict__ q, int32_t d, const uint64_t *__restrict__ topkeys, int64_t nq,
    int32_t ntop, int32_t k, const int32_t *kq, int32_t batch, int32_t beta, float eps,
    const int64_t *__restrict__ perm, const T *__restrict__ raw, int raw_internal,
    int64_t *__restrict__ out_ids, float *__restrict__ out_dist, int32_t *stats, uint32_t *ctr,
    const int32_t *qlist, const uint32_t *qcount, int ip) {
    extern __shared__ float qsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *qs = qsm + warp * (d + d / 4 + 1);  // the query, then its packed bytes
    for (int64_t it = 0;; ++it) {
        int64_t qi;
        if (ctr) {
            uint32_t x = 0;
            if (lane == 0) x = atomicAdd(ctr, 1u);
            qi = __shfl_sync(FULL, x, 0);
            if (qlist) {  // slot x of a list whose length is on the device
                if (qi >= (int64_t)*qcount) break;
                qi = qlist[qi];
            }
        } else {
            if (it > 0) break;
            qi = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
        }
        if (qi >= nq) break;
        rerank_one<R, T>(q, d, topkeys, qi, ntop, k, kq, batch, beta, eps, perm, raw, raw_internal,
                         out_ids, out_dist, stats, qs, ip);
    }
}

template <typename T>
static void launch_rerank_t(const DeviceIndex &ix, const float *q, const uint64_t *topkeys,
                            int64_t nq, int32_t ntop, int32_t k, const int32_t *kq, int32_t batch,
                            int32_t beta, float eps, int64_t *out_ids, float *out_dist,
                            int32_t *stats, int warps, uint32_t *ctr, const int32_t *qlist,
                            const uint32_t *qcount, cudaStream_t st) {
    // persistent: two one-warp CTAs per SM pull queries; else one warp per query
    const dim3 grid(ctr ? (unsigned)std::min<int64_t>(nq, 2 * cur_num_sms())
                        : (unsigned)((nq + warps - 1) / warps));
    if (ctr) FA_CHECK_CUDA(cudaMemsetAsync(ctr, 0, 4, st));
    const int smem = warps * (ix.d + ix.d / 4 + 1) * 4;
    const T *raw = reinterpret_cast<const T *>(ix.raw);
    const int ip = ix.metric == FA_METRIC_IP ? 1 : 0;
#define FA_RR(RR)                                                                                 \
    do {                                                                                          \
        if (ctr) {                                                                                \
            FA_CHECK_CUDA(cudaFuncSetAttribute(k_rerank<RR, T, true>,                             \
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem)); \
            k_rerank<RR, T, true><<<grid, 32 * warps, smem, st>>>(q, ix.d, topkeys, nq, ntop, k, kq, \
                                                                  batch, beta, eps, ix.perm, raw,   \
                                                                  ix.raw_internal,                  \
                                                                  out_ids, out_dist, stats, ctr,    \
                                                                  qlist, qcount, ip);               \
        } else {                                                                                  \
            FA_CHECK_CUDA(cudaFuncSetAttribute(k_rerank<RR, T, false>,                            \
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem)); \
            k_rerank<RR, T, false><<<grid, 32 * warps, smem, st>>>(q, ix.d, topkeys, nq, ntop, k, kq, \
                                                                   batch, beta, eps, ix.perm, raw,  \
                                                                   ix.raw_internal,                 \
                                                                   out_ids, out_dist, stats, ctr,   \
                                                                   nullptr, nullptr, ip);           \
        }                                                                                         \
    } while (0)
    if (k <= 32)
        FA_RR(1);
    else if (k <= 64)
        FA_RR(2);
    else if (k <= 128)
        FA_RR(4);
    else
        FA_REQUIRE(false, FA_ERR_ARG, "re-rank supports k <= 128");
#undef FA_RR
    FA_CHECK_CUDA(cudaGetLastError());
}

// Paged re-rank: persistent one-warp CTAs pull queries; each warp re-reads
// nothing its query already read (its page buffer), and writes the query's
// page-read count. Row ids are caller ids (the pages are laid out by them).
template <int R, typename T>
__global__ void __launch_bounds__(32) k_rerank_paged(
    const float *__restrict__ q, int32_t d, const uint64_t *__restrict__ topkeys, int64_t nq,
    int32_t ntop, int32_t k, const int32_t *kq, int32_t batch, int32_t beta, float eps,
    const int64_t *__restrict__ perm, int64_t *__restrict__ out_ids, float *__restrict__ out_dist,
    int32_t *stats, uint32_t *ctr, PagedCtx base, int64_t cap_pages, int32_t *reads, int ip) {
    extern __shared__ float qsm[];
    const int lane = threadIdx.x & 31;
    PagedCtx pg = base;
    pg.cache = base.cache + (size_t)blockIdx.x * cap_pages * base.page_bytes;
    pg.table = base.table + (size_t)blockIdx.x * base.tsize;
    pg.tslot = base.tslot + (size_t)blockIdx.x * base.tsize;
    for (uint32_t it = 1;; ++it) {
        uint32_t x = 0;
        if (lane == 0) x = atomicAdd(ctr, 1u);
        const int64_t qi = __shfl_sync(FULL, x, 0);
        if (qi >= nq) break;
        pg.gen = it;  // a table entry of an earlier query of this warp reads as empty
        pg.nread = 0;
        rerank_one<R, T>(q, d, topkeys, qi, ntop, k, kq, batch, beta, eps, perm,
                         reinterpret_cast<const T *>(pg.cache), 0, out_ids, out_dist, stats, qsm, ip, &pg);
        if (lane == 0) reads[qi] = pg.nread;
    }
}

void launch_rerank_paged(const DeviceIndex &ix, const float *q, const uint64_t *topkeys, int64_t nq,
                         int32_t ntop, int32_t k, const int32_t *kq, int32_t batch, int32_t beta,
                         float eps, int64_t *out_ids, float *out_dist, int32_t *stats,
                         const PagedBufs &pb, uint32_t *ctr, cudaStream_t st) {
    if (nq == 0) return;
    FA_REQUIRE(ix.vpage && ix.raw, FA_ERR_ARG, "paged re-rank needs paged raw vectors");
    FA_REQUIRE(pb.cap_pages >= ntop, FA_ERR_ARG, "page buffer smaller than the top-n");
    FA_REQUIRE(ix.d % 4 == 0 || ix.raw_dtype == FA_F32, FA_ERR_ARG, "paged re-rank needs d % 4 == 0");
    FA_CHECK_CUDA(cudaMemsetAsync(ctr, 0, 4, st));
    FA_CHECK_CUDA(cudaMemsetAsync(pb.table, 0, sizeof(uint64_t) * (size_t)pb.tsize * pb.warps, st));
    PagedCtx c{};
    c.vpage = ix.vpage;
    c.vslot = ix.vslot;
    c.pages = static_cast<const uint8_t *>(ix.raw);
    c.cache = pb.cache;
    c.table = pb.table;
    c.tslot = pb.tslot;
    c.tsize = pb.tsize;
    c.page_rows = ix.page_rows;
    c.page_bytes = ix.page_bytes;
    const int smem = (ix.d + ix.d / 4 + 1) * 4;
    const int ip = ix.metric == FA_METRIC_IP ? 1 : 0;
#define FA_RRP(RR, TT)                                                                              \
    k_rerank_paged<RR, TT><<<pb.warps, 32, smem, st>>>(q, ix.d, topkeys, nq, ntop, k, kq, batch, beta, \
                                                      eps, ix.perm, out_ids, out_dist, stats, ctr, c,  \
                                                      pb.cap_pages, pb.reads, ip)
#define FA_RRP_T(TT)                                                                               \
    do {                                                                                           \
        if (k <= 32) FA_RRP(1, TT);                                                                \
        else if (k <= 64) FA_RRP(2, TT);                                                           \
        else if (k <= 128) FA_RRP(4, TT);                                                          \
        else FA_REQUIRE(false, FA_ERR_ARG, "re-rank supports k <= 128");                           \
    } while (0)
    if (ix.raw_dtype == FA_U8) FA_RRP_T(uint8_t);
    else if (ix.raw_dtype == FA_I8) FA_RRP_T(int8_t);
    else FA_RRP_T(float);
#undef FA_RRP_T
#undef FA_RRP
    FA_CHECK_CUDA(cudaGetLastError());
}

// warps: queries per CTA. qlist (with ctr): re-rank only queries qlist[0,
// *qcount), the length read on the device. With ctr, a persistent grid of one-warp CTAs (two
// per SM, 64 registers each) pulls queries from the counter: it needs 4096
// registers and 2 d floats of shared memory per SM, so it runs beside a scan
// that fills the SMs, which is how the pipelined search overlaps the two.
void launch_rerank(const DeviceIndex &ix, const float *q, const uint64_t *topkeys, int64_t nq,
                   int32_t ntop, int32_t k, const int32_t *kq, int32_t batch, int32_t beta,
                   float eps, int64_t *out_ids, float *out_dist, int32_t *stats, int warps,
                   uint32_t *ctr, cudaStream_t st, const int32_t *qlist, const uint32_t *qcount) {
    if (nq == 0) return;
    FA_REQUIRE(!qlist || (ctr && warps == 1), FA_ERR_ARG, "a query list needs the persistent form");
    FA_REQUIRE(ix.raw != nullptr, FA_ERR_ARG, "re-rank needs raw vectors in the index");
    if (ix.raw_dtype == FA_U8) {
        FA_REQUIRE(ix.d % 4 == 0, FA_ERR_ARG, "uint8 re-rank needs d % 4 == 0");
        launch_rerank_t<uint8_t>(ix, q, topkeys, nq, ntop, k, kq, batch, beta, eps,
                                 out_ids, out_dist, stats, warps, ctr, qlist, qcount, st);
    } else if (ix.raw_dtype == FA_I8) {
        FA_REQUIRE(ix.d % 4 == 0, FA_ERR_ARG, "int8 re-rank needs d % 4 == 0");
        launch_rerank_t<int8_t>(ix, q, topkeys, nq, ntop, k, kq, batch, beta, eps,
                                out_ids, out_dist, stats, warps, ctr, qlist, qcount, st);
    } else {
        launch_rerank_t<float>(ix, q, topkeys, nq, ntop, k, kq, batch, beta, eps,
                               out_ids, out_dist, stats, warps, ctr, qlist, qcount, st);
    }
}

}  // namespace fa
