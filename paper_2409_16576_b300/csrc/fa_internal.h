// Internal structures of libfa: the device-resident index, per-call
// workspaces and the kernel launch interfaces.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <condition_variable>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fa.h"

namespace fa {

// -------------------------------------------------------------------------
// error plumbing (no exceptions cross the C boundary)
// -------------------------------------------------------------------------
void set_error(const char *fmt, ...);
const char *last_error();

struct Error {
    fa_status st;
    std::string msg;
};

#define FA_CHECK_CUDA(expr)                                                        \
    do {                                                                           \
        cudaError_t _e = (expr);                                                   \
        if (_e != cudaSuccess)                                                     \
            throw ::fa::Error{FA_ERR_CUDA, std::string(#expr) + ": " +             \
                                               cudaGetErrorString(_e)};            \
    } while (0)

#define FA_REQUIRE(cond, status, msg)                                              \
    do {                                                                           \
        if (!(cond)) throw ::fa::Error{(status), std::string(msg)};                \
    } while (0)

// device error flags written by kernels (bit set = condition seen)
enum DevErr : uint32_t {
    DEV_ERR_OVERFLOW = 1u,
    DEV_ERR_TIMEOUT = 2u,
    DEV_ERR_BOUNDS = 4u,
};

// Bytes of one element of a raw vector.
inline int raw_elem(int dt) { return dt == FA_F32 ? 4 : 1; }

// Scan width of M subspaces: the smallest of 8, 16, 32, 48, 64 that holds M.
inline int scan_width(int M) {
    return M <= 8 ? 8 : (M <= 16 ? 16 : (M <= 32 ? 32 : (M <= 48 ? 48 : 64)));
}

// LUT row stride (floats) in shared memory for M subspaces: every position
// p = r + s (r = v mod 32, s < M) must exist, so the row holds M + 31 entries.
inline int lut_row_words(int M) {
    int w = M + 32;
    return w <= 64 ? 64 : (w <= 80 ? 80 : 128);
}

// -------------------------------------------------------------------------
// device index
// -------------------------------------------------------------------------
// Navigation graph of the lists (§4.1 "In-memory Indices"), device copies.
struct ProbeGraph {
    void *heads = nullptr;     // [nlist][d] head vectors (uint8 / int8 / float)
    int32_t head_dtype = FA_F32;
    int32_t *adj = nullptr;    // [nlist][R] out-edges, -1 = none
    int32_t *seeds = nullptr;  // [S] pivot vertices
    float *pivots = nullptr;   // [S][d] their heads as floats (the entry probe's operand)
    // integer heads: the pivots as tensor-core tiles and their squared norms,
    // for an entry probe on the tensor cores (exact: see launch_graph_probe)
    void *pivot_tiles = nullptr;
    float *pivot_norm = nullptr;
    int32_t pivot_kp = 0, pivot_nt = 0;
    int32_t R = 0, S = 0;
};

struct DeviceIndex {
    int64_t n = 0;
    int32_t d = 0, nlist = 0, M = 0, dsub = 0;
    // scan width: M rounded up to 8, 16, 32, 48 or 64 (the scan kernels'
    // widths); the extra subspaces have code 0 and all-zero table rows
    int32_t Mp = 0;
    int32_t metric = FA_METRIC_L2;
    int32_t raw_dtype = FA_U8, raw_location = FA_RAW_NONE;
    int64_t n_rep = 0;        // replica entries
    int64_t n_mem = 0;        // membership table entries
    int64_t max_list = 0;     // longest primary range
    int64_t max_rep = 0;      // longest replica slice

    float *centroids = nullptr;   // [nlist][d]
    float *cnorm = nullptr;       // [nlist] |c|^2
    float *codebooks = nullptr;   // [M][256][dsub]
    uint8_t *codes = nullptr;     // [n_pad][M], internal order, rotated rows
    uint32_t *list_beg = nullptr; // [nlist+1] primary ranges in internal ids
    uint64_t *rep_off = nullptr;  // [nlist+1]
    uint32_t *rep_v = nullptr;    // [n_rep] internal id of each replica entry
    uint32_t *rep_mo = nullptr;   // [n_rep] offset of the vector's membership row
    uint8_t *rep_t = nullptr;     // [n_rep] position of this list in that row (>= 1)
    uint32_t *mem = nullptr;      // [n_mem] membership rows: primary, then replicas
    int64_t *perm = nullptr;      // [n] internal id -> caller id
    const void *raw = nullptr;    // [n][d] raw vectors, device-visible
    int32_t raw_internal = 0;     // rows in internal order (HBM copy) rather than caller order
    void *raw_dev_alloc = nullptr;
    void *raw_host_alloc = nullptr;
    // bf16 operands for the tensor-core paths (allocated on first use)
    void *centroids_bf16 = nullptr; // tensor-core tiles [ntiles][hi, lo][128 x tc_kp]
    int32_t tc_kp = 0, tc_ntiles = 0;
    void *codebooks_bf16 = nullptr; // tensor-core B tiles [M][hi, lo][256 x 16]
    float *cbnorm = nullptr;        // [M][256] |C_m[c]|^2 (FP32)
    float cb_max_norm2 = 0.f;       // largest |C_m[c]|^2 (bounds every table entry)
    uint32_t *lorder = nullptr;     // [nlist] lists by decreasing chunk count (batched form)
    // raw vectors in pages (FA_RAW_HOST_PAGED): page and row of every caller id
    uint32_t *vpage = nullptr;      // [n]
    uint16_t *vslot = nullptr;      // [n]
    int32_t page_rows = 0, page_bytes = 0;  // rows a page, bytes a page (rows x row bytes)
    int64_t n_pages = 0;
    ProbeGraph graph;
    int64_t device_bytes = 0;
    int64_t pinned_bytes = 0;
};

// identity of a captured search (FA_GRAPH): replayed only for an identical call
struct GraphKey {
    const void *q, *oi, *od, *probes, *kq, *npq;
    cudaStream_t st;
    int64_t nq;
    int32_t k, nprobe, lut_prec, lut_gemm, probe_gemm, rerank_n, rerank_batch, rerank_beta;
    int32_t graph_beam, graph_max_check, graph_entry;
    float rerank_eps;
    int32_t flags, threads, ilp, persistent, tile_chunks;
};

// -------------------------------------------------------------------------
// per-call workspace (one slot of the index's pool, §5's per-query blocks)
// -------------------------------------------------------------------------
struct Workspace {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;    // end of the last no-sync call on this slot
    cudaStream_t stream2 = nullptr;  // re-rank stream of the pipelined search (high priority)
    cudaStream_t stream3 = nullptr;  // second scan stream of the pipelined search
    cudaEvent_t fork[8] = {};        // chunk i scanned
    cudaEvent_t lut_done = nullptr, join = nullptr, join3 = nullptr;
    cudaEvent_t marks[5] = {};       // stage boundaries of every call (read by fa_search_trace)
    bool pending = false;
    cudaGraphExec_t gexec = nullptr;  // last captured search (FA_GRAPH)
    GraphKey gkey{};
    int64_t cap_nq = 0;
    int32_t cap_k = 0, cap_nprobe = 0, cap_ntop = 0, cap_lut_bytes = 0;
    float *q = nullptr;            // [cap_nq][d]
    int32_t *probes = nullptr;     // [cap_nq][cap_nprobe]
    int32_t *kq = nullptr;         // [cap_nq]
    int32_t *npq = nullptr;        // [cap_nq]
    int32_t *gentry = nullptr;     // [cap_nq][64] graph walk entry pivots
    int32_t *order = nullptr;      // [cap_nq] scan order
    uint32_t *tchunks = nullptr;   // [cap_nq] chunks per query (tiled form)
    uint32_t *tprefix = nullptr;   // [cap_nq + 1] tiles per query prefix
    uint32_t *tmisc = nullptr;     // [4]: chunks per tile, total chunks (u64)
    uint64_t *partial = nullptr;   // [tile_cap][cap_ntop] per-tile top-n
    int64_t tile_cap = 0;
    uint32_t *bucket = nullptr;    // [nlist] counting-sort buckets
    uint64_t *topkeys = nullptr;   // [cap_nq][cap_ntop]
    int64_t *out_ids = nullptr;    // [cap_nq][cap_k]
    float *out_dist = nullptr;     // [cap_nq][cap_k]
    int32_t *stats = nullptr;      // [cap_nq][4]
    void *lut = nullptr;           // [cap_nq][lut_bytes] global LUT (precision form)
    float *lut_scale = nullptr;    // [cap_nq][2M] per subspace: scale, offset
    float *coarse_d = nullptr;     // coarse distance scratch [coarse_rows][nlist rounded up to 4]
    int64_t coarse_rows = 0;
    uint32_t *err = nullptr;       // device error word
    uint32_t *tile_ctr = nullptr;  // [4] persistent-kernel work counters
    uint64_t *selbuf = nullptr;    // [2 per SM][2 * cap_ntop] keys below the scan's threshold estimate
    int32_t *redo = nullptr;       // [cap_nq] queries the selecting scan hands to the CTA top-n
    // batched form (FA_BATCHED): pairs by list, thresholds, per-query key buffers
    int64_t bq_cap_nq = 0;
    int32_t bq_cap_pairs_np = 0;
    uint32_t bq_cap = 0;
    uint32_t *bq_lcnt = nullptr, *bq_lqoff = nullptr, *bq_lcur = nullptr, *bq_upre = nullptr;
    int32_t *bq_lq = nullptr;      // [cap_nq * cap_nprobe]
    uint32_t *bq_pbits = nullptr;  // [cap_nq][nlist / 32]
    uint64_t *bq_tau = nullptr;    // [cap_nq]
    uint32_t *bq_cnt = nullptr;    // [cap_nq]
    float *bq_qsum = nullptr;      // [cap_nq][2]
    uint64_t *bq_buf = nullptr;    // [cap_nq][bq_cap]
    uint32_t *bq_ctr = nullptr;    // [8]
    // paged re-rank (FA_RAW_HOST_PAGED): per-warp page buffers and page tables
    uint8_t *pg_cache = nullptr;
    uint64_t *pg_table = nullptr;
    uint32_t *pg_tslot = nullptr;
    int32_t *pg_reads = nullptr;   // [cap_nq]
    int64_t pg_cap_pages = 0, pg_cap_nq = 0;
    int32_t pg_tsize = 0, pg_warps = 0;
    // pinned host staging for host-buffer calls
    float *h_q = nullptr;
    int64_t *h_ids = nullptr;
    float *h_dist = nullptr;
    int32_t *h_small = nullptr;    // per-query k / nprobe staging
    uint32_t *h_err = nullptr;
    int32_t *h_stats = nullptr;
    int64_t h_cap_nq = 0;
    int32_t h_cap_k = 0;
};

struct Tune {  // scan launch shape chosen by the autotuner for one class of calls
    int threads = 256, ilp = 1, persistent = 0;
    int tile_chunks = 0;  // > 0: tiled form with tiles of this many 32-candidate chunks
    bool set = false;
};
// class of a call: top-n above 256 (CTA variant) x LUT built in the scan / read from HBM
inline int tune_class(int ntop, bool global_lut) { return (ntop > 256 ? 2 : 0) + (global_lut ? 1 : 0); }

}  // namespace fa

struct fa_index {
    // logical host copies (caller order)
    int64_t n = 0;
    int32_t d = 0, nlist = 0, M = 0;
    int32_t raw_dtype = FA_U8, raw_location = FA_RAW_NONE;
    int32_t metric = FA_METRIC_L2;
    std::vector<float> centroids, codebooks;
    std::vector<uint8_t> codes;
    std::vector<int32_t> primary;
    std::vector<int64_t> rep_off, rep_ids;
    void *h_raw = nullptr;        // caller-order raw copy (pinned when HOST_PINNED)
    bool h_raw_pinned = false;
    void *h_pages = nullptr;      // HOST_PAGED: pinned, mapped pages of rows (§4.3 layout)
    std::vector<int64_t> page_of; // HOST_PAGED: page of each vector (caller ids)
    std::vector<int32_t> slot_of; // HOST_PAGED: row of each vector in its page
    std::vector<int32_t> g_adj, g_seeds;  // navigation graph (host copies), R and S in dev.graph
    int device = 0;
    fa::DeviceIndex dev;
    // workspace pool
    std::mutex mu;
    std::condition_variable cv;
    std::vector<fa::Workspace *> all_ws, free_ws;
    int max_ws = 8;
    std::atomic<int> sticky{0};
    fa::Tune tune[4];  // autotuned scan launch per call class
};

namespace fa {

// -------------------------------------------------------------------------
// host-side building blocks
// -------------------------------------------------------------------------
struct BuildOut {
    float repl_eps = 0.f;  // Eq. 2's epsilon as applied
    std::vector<float> centroids, codebooks;
    std::vector<uint8_t> codes;
    std::vector<int32_t> primary;
    std::vector<int64_t> rep_off, rep_ids;
};

// Trains and encodes (host threads, optionally GPU-assisted).
void train_and_encode(const void *base, int64_t n, int32_t d, fa_dtype dt,
                      const fa_build_params &p, BuildOut &out);

void train_pq_and_encode(const void *base, int64_t n, int32_t d, fa_dtype dt,
                         const fa_build_params &p, const float *X, int64_t S, BuildOut &out);
void encode_with_lists(const void *base, int64_t n, int32_t d, fa_dtype dt,
                       const fa_build_params &p, BuildOut &out);

// Uploads the logical parts to the device (renumbering, rotated codes, CSR).
void upload_index(fa_index *ix);
void free_device_index(fa_index *ix);

// GPU helpers used by the build: nearest-r centroids of rows (float or u8).
void gpu_assign_topr(const void *rows, int64_t n, int32_t d, fa_dtype dt, const float *centroids,
                     int32_t nlist, int32_t r, int32_t *out_ids, float *out_d2);
void gpu_encode(const void *rows, int64_t n, int32_t d, fa_dtype dt, const float *codebooks,
                int32_t M, uint8_t *out_codes);
// Two-level assignment: each row's three nearest of the ntop top-level
// centroids, then its r <= 8 nearest lists among those clusters' lists
// (cluster t holds lists[sub_beg[t] .. sub_beg[t + 1])). out_top (optional)
// receives the nearest cluster.
void gpu_assign_two_level(const void *rows, int64_t n, int32_t d, fa_dtype dt, const float *top,
                          int32_t ntop, const float *lists, int32_t nlist, const int32_t *sub_beg,
                          int32_t r, int32_t *out_ids, float *out_d2, int32_t *out_top);

// -------------------------------------------------------------------------
// kernel launchers (kernels/*.cu)
// -------------------------------------------------------------------------
struct ScanLaunch {
    const float *q;          // [nq][d]
    const int32_t *probes;   // [nq][probe_stride]
    const int32_t *npq;      // [nq] or null (uniform nprobe)
    const int32_t *ntopq;    // [nq] or null (uniform ntop)
    int64_t nq;
    int32_t nprobe, probe_stride, ntop;
    int32_t lut_prec;        // FA_LUT_* of a precomputed global LUT, or -1 to build in smem
    const void *lut;         // global LUT [nq][M][256] (when lut_prec >= 0)
    const float *lut_scale;  // [nq][2M]
    uint64_t *topkeys;       // [nq][ntop] out
    int32_t *stats;          // [nq][4] or null
    uint32_t *err;
    int persistent;
    uint32_t *tile_ctr;
    const int32_t *order;    // [nq] processing order (queries grouped by first probe), or null
    int threads = 256;       // warp-top-n variant: threads per CTA (256 or 512)
    int ilp = 1;             // chunks in flight per warp (1 or 2)
    const uint32_t *tile_prefix = nullptr;  // tiled form: [nq+1] tiles per query prefix
    const uint32_t *tile_T = nullptr;       // chunks per tile (device scalar)
    uint64_t *partial = nullptr;            // [tile capacity][ntop]
    // top-n rows must be sorted ascending (a re-rank that may stop early
    // reads them in order); otherwise a top-n above 256 may be written in
    // any order, valid keys first
    int sorted = 1;
    // top-n above 256, unsorted, one stream: two CTAs per SM keep the keys
    // below a sampled threshold in selbuf and select from there; queries it
    // cannot finish are listed in redo for the one-CTA-per-SM kernel. Needs
    // tile_ctr[0..3] to itself.
    uint64_t *selbuf = nullptr;
    int32_t *redo = nullptr;
    // exhaustive re-rank (Algorithm 1 with eps < 0) fused into the selecting
    // scan: each query's top-k goes straight to out_ids / out_dist (caller
    // ids, sorted); queries handed back keep their top-n row for k_rerank.
    // Needs raw rows in HBM in internal order and k <= 32.
    int fuse_rerank = 0;
    int32_t k = 0, rerank_batch = 32;
    const int32_t *kq = nullptr;
    int64_t *out_ids = nullptr;
    float *out_dist = nullptr;
};


void launch_coarse(const DeviceIndex &ix, const float *q, int64_t nq, int32_t nprobe,
                   int32_t probe_stride, int gemm, Workspace &ws, int32_t *probes,
                   cudaStream_t st);
int coarse_launches(const DeviceIndex &ix, int64_t nq, int gemm, const Workspace &ws);
void prepare_centroid_tiles(const float *cent, int32_t nlist, int32_t d, std::vector<uint16_t> &out,
                            int32_t &Kp, int32_t &ntiles);
void prepare_codebook_tiles(const float *cb, int32_t M, int32_t d, std::vector<uint16_t> &tiles,
                            std::vector<float> &norms);
int64_t coarse_tc_ldd(int32_t nlist);
void launch_coarse_tc(const DeviceIndex &ix, const float *q, int64_t rows, int32_t ntop, float *D,
                      int32_t *probes, int32_t probe_stride, uint32_t *err, cudaStream_t st);
void launch_query_order(const int32_t *probes, int64_t nq, int32_t stride, int32_t nlist,
                        uint32_t *cnt, int32_t *order, cudaStream_t st);
void launch_tile_plan(const DeviceIndex &ix, const int32_t *probes, const int32_t *npq, int64_t nq,
                      int32_t nprobe, int32_t stride, uint32_t T_req, uint32_t cap,
                      uint32_t *chunks, unsigned long long *total, uint32_t *T_out,
                      uint32_t *prefix, cudaStream_t st);
void launch_tile_merge(const uint64_t *partial, const uint32_t *prefix, int64_t nq, int32_t ntop,
                       uint64_t *topkeys, cudaStream_t st);
// Returns true when the exhaustive re-rank ran fused in the scan (outputs
// written for every query the selecting scan finished; the rest are listed
// in ScanLaunch::redo, their count in tile_ctr[3]).
bool launch_scan(const DeviceIndex &ix, const ScanLaunch &a, cudaStream_t st);
// Buffers of the batched form (list-major scan over the whole batch).
struct BatchBufs {
    uint32_t *lcnt, *lqoff, *lcur, *upre, *pbits, *cnt, *ctr;
    int32_t *lq;
    uint64_t *tau, *buf;
    float *qsum;
    uint32_t cap;          // keys per query buffer
    uint32_t tile_chunks;  // chunks per unit of a long list
    int64_t qsub;          // queries per sub-batch
};
// Batched form of launch_scan (FP16 table with one scale per query): the
// same results contract, the same redo list and fused re-rank.
bool launch_batched(const DeviceIndex &ix, const ScanLaunch &a, const BatchBufs &bb, cudaStream_t st);
// Standard deviations of the CTA top-n threshold estimate (test hook).
void set_tau_sigma(float sigma);
void launch_wait_nothing(uint32_t polls, const uint32_t *flag, uint32_t *err, cudaStream_t st);
// true when an injected allocation failure (fa_debug_fail_alloc) is due now
bool alloc_fault();
// uniform != 0: one scale per query for all subspaces (the batched form sums
// the stored entries directly)
void launch_lut_global(const DeviceIndex &ix, const float *q, int64_t nq, int prec, int gemm,
                       void *lut, float *lut_scale, uint32_t *err, cudaStream_t st, int uniform = 0);
void launch_finish(const DeviceIndex &ix, const uint64_t *topkeys, int64_t nq, int32_t ntop,
                   int32_t k, const int32_t *kq, int64_t *out_ids, float *out_dist,
                   cudaStream_t st);
// Paged re-rank buffers (one page buffer and page table per warp).
struct PagedBufs {
    uint8_t *cache;
    uint64_t *table;
    uint32_t *tslot;
    int32_t *reads;         // [nq] pages each query read
    int64_t cap_pages;      // pages a warp's buffer holds (>= top-n)
    int32_t tsize, warps;   // table entries a warp (power of two), warps of the grid
};
void launch_rerank_paged(const DeviceIndex &ix, const float *q, const uint64_t *topkeys, int64_t nq,
                         int32_t ntop, int32_t k, const int32_t *kq, int32_t batch, int32_t beta,
                         float eps, int64_t *out_ids, float *out_dist, int32_t *stats,
                         const PagedBufs &pb, uint32_t *ctr, cudaStream_t st);
// Coarse probe by the navigation graph: probes [nq][probe_stride], lists
// found per query in npq_out (npq_in: optional per-query target).
// entry < S: each walk starts from the entry pivots nearest its query (an
// exact probe of the pivots in scratch, then entry_buf [nq][entry]); entry
// == S: from every pivot.
void launch_graph_probe(const DeviceIndex &ix, const float *q, int64_t nq, int32_t nprobe,
                        int32_t probe_stride, int32_t beam, int32_t max_check, int32_t entry,
                        const int32_t *npq_in, int32_t *probes, int32_t *npq_out, int32_t *checks,
                        float *scratch, int64_t scratch_rows, int32_t *entry_buf, uint32_t *err,
                        cudaStream_t st);
// rows x centroids -> top-ntop columns per row (FP32 direct differences, or -<x, c>)
void launch_l2_topn(const float *X, int64_t nx, int32_t d, const float *C, int32_t nc, int32_t ntop,
                    float *scratch, int64_t scratch_rows, int32_t *out_ids, int32_t out_stride,
                    cudaStream_t st, int ip);
int graph_table_bits(int32_t max_check, int32_t R, int32_t S);
// Storage layout of §4.3 for vectors of the given primary lists.
int64_t page_layout(const std::vector<int32_t> &primary, int32_t nlist, int32_t cap,
                    std::vector<int64_t> &page_of, std::vector<int32_t> &slot_of);
void launch_rerank(const DeviceIndex &ix, const float *q, const uint64_t *topkeys, int64_t nq,
                   int32_t ntop, int32_t k, const int32_t *kq, int32_t batch, int32_t beta,
                   float eps, int64_t *out_ids, float *out_dist, int32_t *stats, int warps,
                   uint32_t *ctr, cudaStream_t st, const int32_t *qlist = nullptr,
                   const uint32_t *qcount = nullptr);
void launch_debug_candidates(const DeviceIndex &ix, const int32_t *probes, int32_t nprobe,
                             uint32_t *out, uint32_t *count, uint32_t cap, cudaStream_t st);

int num_sms(int device);
// SM count of the current device (every launch runs with the index's device current)
int cur_num_sms();

}  // namespace fa
