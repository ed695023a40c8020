// Coarse probe by the navigation graph (§3 step 2, §4.1 "In-memory
// Indices"): the lists are the vertices of a graph, each with a head vector,
// and a query walks it best first to find its top-m lists.
//
// The walk (the same steps as the oracle's, so that the two agree list for
// list): every seed is evaluated (every pivot vertex, or the entry pivots
// nearest the query, found first by an exact probe of the pivots' heads, in
// the spirit of the tree SPTAG starts its graph search from); then, while
// fewer than max_check vertices
// were checked and the beam (the L best (distance, id) pairs seen) holds an
// unexpanded vertex, the first such vertex is expanded and its unseen
// out-neighbours are evaluated. The top-m lists are the beam's first m.
//
// One warp per query:
//   * the beam lives in registers as a warp-wide sorted list of 32*RB keys
//     (distance, id), truncated to L after every merge;
//   * the seen set is an open-addressing table in shared memory (entries
//     id + 1, bit 31 = expanded), sized to twice the most vertices a walk can
//     check, so a probe sequence always ends;
//   * an expansion evaluates the (up to 32) out-neighbours of a vertex
//     together: one lane per neighbour claims it in the table (atomicCAS, so
//     a vertex is evaluated once), the rows are read by the re-rank's
//     row-distance routine (eight lanes a row, 16-byte pieces), and the
//     sorted batch is merged into the beam. The beam after a batch is the L
//     smallest of the old beam and the batch, whatever the order inside it,
//     which is what the oracle's one-at-a-time insertion leaves too.
//
// Integer heads (uint8 / int8 vectors) with an integral query give exact
// distances (every term and partial sum is an integer below 2^24), so the
// walk's decisions equal the FP64 oracle's.
#include "../fa_internal.h"
#include "rerank_rows.cuh"
#include "warp_topk.cuh"

namespace fa {

namespace {

struct GraphArgs {
    const float *q;
    int64_t nq;
    int32_t d;
    const void *heads;  // [nlist][d] of the head type
    const int32_t *adj; // [nlist][R], -1 = no edge
    int32_t R;
    const int32_t *seeds;   // pivot vertices
    int32_t S;              // seeds a walk starts from
    const int32_t *qseeds;  // optional [nq][S]: each query's own pivots (indices into seeds)
    int32_t L, max_check, nprobe, probe_stride;
    const int32_t *npq_in;  // optional per-query list count (clamped to 1..nprobe)
    int32_t *probes;        // [nq][probe_stride]
    int32_t *npq_out;       // lists found per query (the scan's per-query nprobe)
    int32_t *checks;        // optional [nq]: vertices checked
    int32_t hbits;          // table entries = 1 << hbits
    int ip;
};

constexpr uint32_t EXPANDED = 0x80000000u;

// Claims vertex v in the seen table: true when this call inserted it.
__device__ __forceinline__ bool seen_claim(uint32_t *tab, int32_t hbits, uint32_t v) {
    const uint32_t mask = (1u << hbits) - 1u;
    uint32_t h = (v * 2654435761u) >> (32 - hbits);
    for (uint32_t i = 0; i <= mask; ++i) {
        const uint32_t old = atomicCAS(&tab[h], 0u, v + 1u);
        if (old == 0u) return true;
        if ((old & ~EXPANDED) == v + 1u) return false;
        h = (h + 1u) & mask;
    }
    return false;  // not reached: the table holds at most half its size
}

// Entry of a vertex already in the table.
__device__ __forceinline__ uint32_t seen_slot(const uint32_t *tab, int32_t hbits, uint32_t v) {
    const uint32_t mask = (1u << hbits) - 1u;
    uint32_t h = (v * 2654435761u) >> (32 - hbits);
    for (uint32_t i = 0; i <= mask; ++i) {
        if ((tab[h] & ~EXPANDED) == v + 1u) return h;
        h = (h + 1u) & mask;
    }
    return 0u;  // not reached: beam vertices are in the table
}

template <int RB, typename T>
__global__ void __launch_bounds__(32) k_graph_probe(GraphArgs a) {
    extern __shared__ uint32_t gsm[];
    const int lane = threadIdx.x;
    const int64_t qi = blockIdx.x;
    uint32_t *tab = gsm;
    float *qs = reinterpret_cast<float *>(gsm + (1u << a.hbits));
    uint32_t *qp = reinterpret_cast<uint32_t *>(qs + a.d);
    for (uint32_t i = lane; i < (1u << a.hbits); i += 32) tab[i] = 0u;
    for (int j = lane; j < a.d; j += 32) qs[j] = a.q[qi * a.d + j];
    __syncwarp();
    bool qint = false;
    if (!a.ip && std::is_same<T, uint8_t>::value && a.d <= 258 && a.d % 16 == 0) qint = pack_u8_query(qs, a.d, qp);
    __syncwarp();
    const T *heads = static_cast<const T *>(a.heads);
    uint64_t Q[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) Q[r] = KEY_INF;
    int32_t checks = 0;

    // evaluates the vertices the lanes hold (v < 0: none) and offers them to the beam
    auto offer = [&](int64_t v) {
        checks += __popc(__ballot_sync(FULL, v >= 0));
        const float dist = exact_rows_any<T>(heads, a.d, qs, qp, qint, v, a.ip != 0);
        uint64_t key[1] = {v >= 0 ? make_key(dist, (uint32_t)v) : KEY_INF};
        const uint64_t last = warp_elem<RB>(Q, a.L - 1);
        if (__ballot_sync(FULL, key[0] < last)) {
            bitonic_sort<1>(key);
            merge_sorted32<RB>(Q, key[0]);
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (r * 32 + lane >= a.L) Q[r] = KEY_INF;
        }
    };

    for (int s0 = 0; s0 < a.S; s0 += 32) {
        int32_t v = -1;
        if (s0 + lane < a.S) v = a.qseeds ? a.seeds[a.qseeds[qi * a.S + s0 + lane]] : a.seeds[s0 + lane];
        const bool fresh = v >= 0 && seen_claim(tab, a.hbits, (uint32_t)v);
        __syncwarp();
        offer(fresh ? v : -1);
    }
    while (checks < a.max_check) {
        // the first vertex of the beam not yet expanded
        int32_t p = -1;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            if (p >= 0) continue;  // (uniform across the warp)
            const uint32_t id = (uint32_t)(Q[r] & 0xffffffffu);
            uint32_t slot = 0;
            bool open = false;
            if (Q[r] != KEY_INF) {
                slot = seen_slot(tab, a.hbits, id);
                open = (tab[slot] & EXPANDED) == 0u;
            }
            const uint32_t m = __ballot_sync(FULL, open);
            if (m) {
                const int src = __ffs(m) - 1;
                if (lane == src) tab[slot] |= EXPANDED;
                p = (int32_t)__shfl_sync(FULL, id, src);
            }
        }
        if (p < 0) break;
        __syncwarp();
        const int32_t *nb = a.adj + (int64_t)p * a.R;
        for (int e0 = 0; e0 < a.R; e0 += 32) {
            const int32_t u = e0 + lane < a.R ? nb[e0 + lane] : -1;
            const bool fresh = u >= 0 && seen_claim(tab, a.hbits, (uint32_t)u);
            __syncwarp();
            offer(fresh ? u : -1);
        }
    }
    int cnt = 0;
#pragma unroll
    for (int r = 0; r < RB; ++r) cnt += __popc(__ballot_sync(FULL, Q[r] != KEY_INF));
    int want = a.npq_in ? a.npq_in[qi] : a.nprobe;
    want = want < 1 ? 1 : (want > a.nprobe ? a.nprobe : want);
    const int m = cnt < want ? cnt : want;
    int32_t *row = a.probes + qi * a.probe_stride;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        const int e = r * 32 + lane;
        if (e < a.nprobe) row[e] = e < m ? (int32_t)(Q[r] & 0xffffffffu) : -1;
    }
    for (int e = 32 * RB + lane; e < a.nprobe; e += 32) row[e] = -1;
    if (lane == 0) {
        a.npq_out[qi] = m;
        if (a.checks) a.checks[qi] = checks;
    }
}

}  // namespace

int graph_table_bits(int32_t max_check, int32_t R, int32_t S) {
    const int64_t most = std::max<int64_t>(S, (int64_t)max_check + R);
    int bits = 6;
    while ((1ll << bits) < 2 * most) ++bits;
    return bits;
}

void launch_graph_probe(const DeviceIndex &ix, const float *q, int64_t nq, int32_t nprobe,
                        int32_t probe_stride, int32_t beam, int32_t max_check, int32_t entry,
                        const int32_t *npq_in, int32_t *probes, int32_t *npq_out, int32_t *checks,
                        float *scratch, int64_t scratch_rows, int32_t *entry_buf, uint32_t *err,
                        cudaStream_t st) {
    if (nq == 0) return;
    const ProbeGraph &g = ix.graph;
    FA_REQUIRE(g.adj && g.heads, FA_ERR_ARG, "the index has no navigation graph");
    FA_REQUIRE(beam >= nprobe && beam <= 256, FA_ERR_ARG, "graph beam must be in nprobe..256");
    FA_REQUIRE(max_check >= 0, FA_ERR_ARG, "graph max_check < 0");
    FA_REQUIRE(entry >= 1 && entry <= g.S, FA_ERR_ARG, "graph entry must be in 1..S");
    const bool per_query = entry < g.S;
    if (per_query) {
        // the entry pivots nearest each query, ties by pivot order. Integer
        // heads: on the tensor cores (bf16 holds them exactly, and for an
        // integral query every product, norm and sum is an integer below
        // 2^24, so the distances are exact); else FP32 direct differences.
        FA_REQUIRE(entry <= 64 && entry_buf && scratch, FA_ERR_ARG, "graph entry above 64");
        if (g.pivot_tiles) {
            DeviceIndex P = ix;
            P.centroids_bf16 = g.pivot_tiles;
            P.cnorm = g.pivot_norm;
            P.nlist = g.S;
            P.tc_kp = g.pivot_kp;
            P.tc_ntiles = g.pivot_nt;
            for (int64_t r0 = 0; r0 < nq; r0 += scratch_rows) {
                const int64_t rows = std::min<int64_t>(scratch_rows, nq - r0);
                launch_coarse_tc(P, q + r0 * ix.d, rows, entry, scratch, entry_buf + r0 * entry, entry, err, st);
            }
        } else {
            launch_l2_topn(q, nq, ix.d, g.pivots, g.S, entry, scratch, scratch_rows, entry_buf, entry, st,
                           ix.metric == FA_METRIC_IP ? 1 : 0);
        }
    }
    const int32_t S = per_query ? entry : g.S;
    const int hbits = graph_table_bits(max_check, g.R, S);
    const size_t smem = (sizeof(uint32_t) << hbits) + sizeof(float) * (ix.d + ix.d / 4 + 1);
    FA_REQUIRE(smem <= 200 * 1024, FA_ERR_ARG, "graph max_check too large for the seen table");
    GraphArgs a{};
    a.q = q;
    a.nq = nq;
    a.d = ix.d;
    a.heads = g.heads;
    a.adj = g.adj;
    a.R = g.R;
    a.seeds = g.seeds;
    a.S = S;
    a.qseeds = per_query ? entry_buf : nullptr;
    a.L = beam;
    a.max_check = max_check;
    a.nprobe = nprobe;
    a.probe_stride = probe_stride;
    a.npq_in = npq_in;
    a.probes = probes;
    a.npq_out = npq_out;
    a.checks = checks;
    a.hbits = hbits;
    a.ip = ix.metric == FA_METRIC_IP ? 1 : 0;
    FA_REQUIRE(nq <= 0x7fffffffll, FA_ERR_ARG, "too many queries for one graph probe launch");
#define FA_GP(RB, TT)                                                                                   \
    do {                                                                                                \
        FA_CHECK_CUDA(cudaFuncSetAttribute(k_graph_probe<RB, TT>,                                      \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));   \
        k_graph_probe<RB, TT><<<(unsigned)nq, 32, smem, st>>>(a);                                      \
    } while (0)
#define FA_GP_T(TT)                                                                                     \
    do {                                                                                                \
        if (beam <= 32) FA_GP(1, TT);                                                                   \
        else if (beam <= 64) FA_GP(2, TT);                                                              \
        else if (beam <= 128) FA_GP(4, TT);                                                             \
        else FA_GP(8, TT);                                                                              \
    } while (0)
    if (g.head_dtype == FA_U8) FA_GP_T(uint8_t);
    else if (g.head_dtype == FA_I8) FA_GP_T(int8_t);
    else FA_GP_T(float);
#undef FA_GP_T
#undef FA_GP
    FA_CHECK_CUDA(cudaGetLastError());
}

}  // namespace fa
