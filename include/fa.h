/*
 * fa.h - C ABI of a B300 (sm_103a) implementation of the GPU filtering path of
 * FusionANNS-style IVF-PQ search (Tian et al., "FusionANNS", arXiv 2409.16576).
 *
 * The path for one query (the online steps of Section 3):
 *   coarse probe  the nprobe posting lists nearest to the query (step 2; the
 *                 paper walks an in-memory graph, this library computes the
 *                 exact top-nprobe on the GPU)
 *   LUT           dist(q_i, c) for every subspace i and centroid c (step 1)
 *   gather        the vector ids of the probed lists (steps 3-4)
 *   dedup         every distinct id once (step 5)
 *   ADC           Eq. 1 over the uint8 PQ codes held in HBM (step 6)
 *   top-n         the n smallest ADC distances (step 7)
 *   re-rank       optional, Algorithm 1 / Eq. 3 on exact distances over raw
 *                 vectors held in pinned host memory or HBM (step 8, §4.2)
 *
 * Conventions shared by every call:
 *   - Distances are squared L2 (the form of Eq. 1 that splits into a sum over
 *     subspaces). Without re-rank they are ADC distances; with re-rank they
 *     are exact FP32 distances on the raw vectors.
 *   - Result rows are row-major [nq][k], ascending by (distance, id); ids are
 *     the caller's 0-based vector ids. A query with fewer than k distinct
 *     candidates gets rows padded with id -1 and distance +inf.
 *   - The caller owns every buffer it passes; the library copies what it keeps.
 *     The library owns the index (host copies, device memory, pinned memory).
 *   - Functions return fa_status and never throw across this boundary. After a
 *     failure the outputs are undefined; fa_last_error() gives a message
 *     (per calling thread). A CUDA error that leaves the context unusable marks
 *     the index FA_ERR_STATE for every later call.
 *   - fa_search / fa_search_ex may be called from several host threads on one
 *     index at once; each call takes a workspace slot from the index's pool.
 *   - Every device-side wait is bounded; exceeding a bound returns
 *     FA_ERR_TIMEOUT, an internal capacity overflow returns FA_ERR_OVERFLOW.
 */
#ifndef FA_H
#define FA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fa_index fa_index; /* opaque, owned by the library */

typedef enum fa_status {
    FA_OK = 0,
    FA_ERR_ARG = 1,      /* an argument is out of range or inconsistent */
    FA_ERR_OOM = 2,      /* device or host allocation failed */
    FA_ERR_CUDA = 3,     /* a CUDA call failed */
    FA_ERR_TIMEOUT = 4,  /* a bounded device-side wait ran out */
    FA_ERR_OVERFLOW = 5, /* an internal buffer bound was exceeded */
    FA_ERR_STATE = 6,    /* the index is unusable after an earlier fatal error */
    FA_ERR_BUSY = 7,     /* non-blocking admission found no free slot */
    FA_ERR_IO = 8,       /* file read/write failed (save/load) */
    FA_ERR_NODEV = 9     /* no usable CUDA device */
} fa_status;

/* Element type of base and raw vectors: float32, uint8 (SIFT-like) or int8
 * (SPACEV-like, Table 1). Queries are always float32. */
typedef enum fa_dtype { FA_F32 = 0, FA_U8 = 1, FA_I8 = 2 } fa_dtype;

/* Where the raw vectors used by the re-rank live. The paper keeps them on SSD
 * (§4.1 "Raw Vectors on SSDs"); pinned host memory read by the GPU over the
 * host link stands in for that tier. */
typedef enum fa_raw_location {
    FA_RAW_NONE = 0,
    FA_RAW_HOST_PINNED = 1,
    FA_RAW_DEVICE = 2,
    /* pinned host memory in 4 KB pages with the storage layout of §4.3: each
     * list's primary members form a bucket, buckets fill pages of their own
     * and their unaligned tails share pages by a max-min rule. The re-rank
     * then reads whole pages: a mini-batch reads each distinct page once
     * (intra-mini-batch merge) and skips the pages the query read in earlier
     * mini-batches, which a per-query page buffer in HBM holds
     * (inter-mini-batch deduplication); a row is read from that buffer. */
    FA_RAW_HOST_PAGED = 3
} fa_raw_location;

/* Distance of the search. L2: squared L2 (Eq. 1 as the paper writes it). IP:
 * the negated inner product -<q, x>, which also splits over subspaces, so
 * the table entries are -<q_m, C_m[c]>, the coarse probe ranks lists by
 * -<q, c> and the re-rank uses the exact -<q, x>; the lists themselves come
 * from L2 k-means either way (the SPACEV-like workload's second metric). */
typedef enum fa_metric { FA_METRIC_L2 = 0, FA_METRIC_IP = 1 } fa_metric;

/* Storage precision of the per-query lookup table (step 1). The scan always
 * accumulates in FP32; F16 and FP8 (e4m3) tables carry a per-query scale and
 * a per-subspace offset. */
typedef enum fa_lut_prec { FA_LUT_F32 = 0, FA_LUT_F16 = 1, FA_LUT_FP8 = 2 } fa_lut_prec;

/* How the LUT (step 1) and the coarse probe (step 2) are computed.
 *   FA_GEMM_SIMT_F32  FP32 direct differences on the CUDA cores; for the LUT
 *                     this is built straight into the scan CTA's shared memory.
 *   FA_GEMM_BF16_TC   the expanded form |q|^2 - 2 q.c + |c|^2 with the dot
 *                     products on the tcgen05 tensor cores (BF16 operands,
 *                     FP32 accumulation in tensor memory). */
typedef enum fa_gemm { FA_GEMM_SIMT_F32 = 0, FA_GEMM_BF16_TC = 1 } fa_gemm;

/* probe_gemm may also name the navigation graph (§3 step 2, §4.1 "In-memory
 * Indices"): the top-nprobe lists come from a best-first walk over the
 * index's list graph (fa_build_probe_graph) instead of the exact distances
 * to every centroid, and the LUT (step 1) is built at the same time on a
 * second stream, as the paper overlaps steps 1 and 2. A query whose walk
 * finds fewer than nprobe lists scans the ones it found. */
#define FA_PROBE_GRAPH 2

/* ------------------------------------------------------------------------- */
/* Index build (offline processing of Section 3, multi-tiered index of §4.1) */
/* ------------------------------------------------------------------------- */

typedef struct fa_build_params {
    int32_t nlist;             /* posting lists (IVF cells), >= 1 */
    int32_t M;                 /* PQ subspaces; d % M == 0, d / M <= 16, M <= 64 (the
                                * scans run 8, 16, 32, 48 or 64 subspaces; a
                                * smaller M is padded with subspaces whose codes
                                * and table entries are 0) */
    int32_t kmeans_iters;      /* Lloyd iterations of the coarse and PQ k-means */
    int32_t max_lists_per_vec; /* Eq. 2 cap on lists per vector, 1..8 */
    int64_t train_sample;      /* rows sampled for training; 0 = automatic */
    uint64_t seed;             /* seed of every random choice of the build */
    float repl_eps;            /* Eq. 2 epsilon; 0 = each vector in one list; < 0 =
                                * chosen by bisection so that a vector joins
                                * -repl_eps lists on average (e.g. -1.08) */
    int32_t raw_location;      /* fa_raw_location: keep raw vectors for re-rank */
    int32_t use_gpu;           /* 1 = run assignment and encoding on the GPU */
    int32_t metric;            /* fa_metric of the searches on this index */
} fa_build_params;

/* Fills p with defaults: nlist 256, M 16, 10 iterations, 1 list per vector,
 * automatic sample, seed 20240916, no replication, raw vectors not kept,
 * GPU-assisted build. */
void fa_build_params_init(fa_build_params *p);

/* Trains an IVF-PQ index on n host vectors base[n][d] of type dt and uploads
 * it to the current CUDA device: coarse k-means (nlist centroids), Eq. 2
 * boundary replication (a vector joins every list C_i with
 * |v - C_i| <= (1 + repl_eps) |v - C_1|, at most max_lists_per_vec lists),
 * PQ training (M sub-codebooks of 256 centroids over contiguous blocks of
 * d/M coordinates, §2.2) and encoding. n must be below 2^32. With use_gpu and
 * nlist >= 32768 the lists come from two-level k-means (about sqrt(nlist)
 * top-level clusters, each split into its share of the lists, as the paper's
 * hierarchical clustering of §4.1), and a vector's lists are looked up among
 * the lists of its three nearest top-level clusters.
 * Returns FA_ERR_ARG for bad shapes, FA_ERR_OOM / FA_ERR_CUDA on failure. */
fa_status fa_build_index(const void *base, int64_t n, int32_t d, fa_dtype dt,
                         const fa_build_params *p, fa_index **out);

/* Builds an index whose posting lists the caller already has: centroids
 * [nlist][d] and the list of every vector, primary[n] (no coarse k-means, no
 * replication). Only the PQ sub-codebooks are trained (on a sample) and every
 * vector encoded, as in fa_build_index; p->nlist is ignored. */
fa_status fa_build_index_lists(const void *base, int64_t n, int32_t d, fa_dtype dt,
                               const float *centroids, int32_t nlist, const int32_t *primary,
                               const fa_build_params *p, fa_index **out);

/* The logical content of an index. Every pointer is host memory. */
typedef struct fa_index_parts {
    int64_t n;                /* vectors */
    int32_t d;                /* dimension */
    int32_t nlist;            /* posting lists */
    int32_t M;                /* subspaces (d % M == 0) */
    int32_t raw_dtype;        /* fa_dtype of raw */
    int32_t raw_location;     /* fa_raw_location */
    int32_t pad0;
    const float *centroids;   /* [nlist][d] list centroids */
    const float *codebooks;   /* [M][256][d/M] PQ sub-codebooks */
    const uint8_t *codes;     /* [n][M] PQ code of each vector */
    const int32_t *primary;   /* [n] the list each vector belongs to first */
    const int64_t *rep_off;   /* [nlist+1] replica slice offsets, or NULL */
    const int64_t *rep_ids;   /* [rep_off[nlist]] replicated vector ids */
    const void *raw;          /* [n][d] raw vectors, or NULL */
    int32_t metric;           /* fa_metric */
    int32_t pad1;
} fa_index_parts;

/* Builds an index from given parts (no training): list l holds the vectors
 * whose primary list is l followed by rep_ids[rep_off[l] .. rep_off[l+1]).
 * A vector may appear in a list at most once. The library copies every array.
 * Returns FA_ERR_ARG for an inconsistent description. */
fa_status fa_index_from_parts(const fa_index_parts *parts, fa_index **out);

/* A read-only view of the index's host copies (valid until fa_free_index). */
fa_status fa_index_get_parts(const fa_index *ix, fa_index_parts *out);

typedef struct fa_index_info {
    int64_t n, n_rep_entries, max_list_len, max_rep_len;
    int64_t device_bytes, pinned_bytes;
    int32_t d, nlist, M, device;
} fa_index_info;

fa_status fa_index_info_get(const fa_index *ix, fa_index_info *out);

/* Checkpoint: a versioned binary file holding the parts of the index. */
fa_status fa_save_index(const fa_index *ix, const char *path);
fa_status fa_load_index(const char *path, int32_t raw_location, fa_index **out);

void fa_free_index(fa_index *ix);

/* ------------------------------------------------------------------------- */
/* Search                                                                    */
/* ------------------------------------------------------------------------- */

/* flags of fa_search_params */
#define FA_QUERIES_ON_DEVICE 0x1 /* queries is a device pointer */
#define FA_OUTPUTS_ON_DEVICE 0x2 /* out_ids / out_dist are device pointers */
#define FA_NONBLOCKING 0x4       /* FA_ERR_BUSY instead of waiting for a slot */
#define FA_PERSISTENT 0x8        /* batching form: persistent CTAs over tiles of
                                  * uneven queries (top-n <= 256) */
#define FA_NO_SYNC 0x10          /* return without synchronizing sp->stream
                                  * (device outputs only) */
#define FA_GRAPH 0x20            /* capture the call's kernels into a CUDA graph
                                  * on first use and replay it on later calls
                                  * with the same shape, parameters, pointers
                                  * and stream (device queries and outputs, no
                                  * stats or trace) */
#define FA_SERIAL 0x40           /* re-rank the whole batch after the whole scan.
                                  * By default a call of >= 4096 queries that
                                  * re-ranks from host memory is cut into chunks:
                                  * chunk i's re-rank (a second stream of the
                                  * library's, waiting on the host link) runs
                                  * while chunk i+1 is scanned, as the paper's
                                  * concurrent queries (one CPU thread each,
                                  * §5) overlap one query's re-rank with
                                  * another's GPU filtering.
                                  * The results are the same either way. */
#define FA_BATCHED 0x80          /* batched form: the whole batch is scanned list
                                  * by list. The (query, probed list) pairs are
                                  * grouped by list; the queries that probe a
                                  * list share each 32-bit word of a shared-
                                  * memory table (two FP16 or four FP8 entries),
                                  * so one lookup per code byte serves two or
                                  * four queries, and a list's codes are read
                                  * once for all of them. Needs lut_prec
                                  * FA_LUT_F16 or FA_LUT_FP8; the table then
                                  * carries one scale per query (fa_debug_lut
                                  * with this flag returns that table). FP16
                                  * entries are summed in FP32; FP8 entries in
                                  * half2 over 16 subspaces, then in FP32.
                                  * Workspace: a key buffer of max(4 top-n,
                                  * 65536) keys (8 bytes each) per query of
                                  * the call, so split very large batches;
                                  * FA_ERR_OOM when it does not fit. */

/* Optional per-call trace, measured with CUDA events on the call's stream
 * (ms of device time per stage; launches = kernels this call launched). An
 * exhaustive re-rank (rerank_eps < 0, k <= 32) of uint8 raw rows held in HBM
 * runs inside the scan kernel for a top-n above 256, so its time is then part
 * of scan_ms and post_ms covers only the queries the scan handed back. */
typedef struct fa_search_trace {
    float coarse_ms, lut_ms, scan_ms, post_ms, total_ms;
    int32_t launches;
    int32_t handed_back;  /* queries the selecting or batched scan handed back to
                             the per-query scan (0 on the other paths) */
} fa_search_trace;

typedef struct fa_search_params {
    int32_t lut_prec;     /* fa_lut_prec */
    int32_t lut_gemm;     /* fa_gemm for the LUT */
    int32_t probe_gemm;   /* fa_gemm for the coarse probe */
    int32_t rerank_n;     /* 0: ADC top-k. >0: re-rank the ADC top-rerank_n (<= 16384;
                           * above 4096 the scan needs the top-n beside the LUT in
                           * shared memory, so large M may return FA_ERR_ARG) */
    int32_t rerank_batch; /* Algorithm 1 BatchSize, 1..4096 */
    int32_t rerank_beta;  /* Algorithm 1 beta (>= 1) */
    float rerank_eps;     /* Algorithm 1 epsilon (< 0: never stop early) */
    int32_t flags;        /* FA_* flags above */
    const int32_t *k_per_query;      /* optional [nq]; each <= k */
    const int32_t *nprobe_per_query; /* optional [nq]; each clamped to [1, nprobe] */
    const int32_t *probes;           /* optional [nq][nprobe] given probe lists */
    void *stream;                    /* cudaStream_t to run on, or NULL */
    int64_t *stats;                  /* optional host [nq][4]: gathered ids,
                                        distinct ids, re-rank mini-batches run,
                                        candidates handed to the re-rank */
    fa_search_trace *trace;          /* optional host trace (forces a sync) */
    int32_t *page_reads;             /* optional host [nq]: pages each query's re-rank
                                        read (raw vectors in FA_RAW_HOST_PAGED) */
    int32_t graph_beam;              /* FA_PROBE_GRAPH: beam, nprobe..256 (0: min(256, 2 nprobe)) */
    int32_t graph_max_check;         /* FA_PROBE_GRAPH: expansions start only while fewer
                                        vertices were checked (0: 16 nprobe + entry) */
    int32_t graph_entry;             /* FA_PROBE_GRAPH: the walk starts from the graph_entry
                                        pivots nearest the query (exact probe of the pivots;
                                        0: 16; >= S: from every pivot; else <= 64) */
} fa_search_params;

/* Fills sp with the plain FP32 form: F32 LUT built in the scan CTA, FP32 coarse
 * probe, no re-rank (BatchSize 32, beta 2, eps 0 when enabled), no flags. */
void fa_search_params_init(fa_search_params *sp);

/* Top-k search for nq host queries[nq][d] (float32) with the plain FP32 form.
 * out_ids [nq][k] and out_dist [nq][k] are host buffers. nprobe is clamped to
 * [1, nlist]. nq == 0 returns FA_OK. d must equal the index's d, 1 <= k <= 16384
 * (k <= 128 when re-ranking; k above 4096 needs the top-k beside the LUT in
 * shared memory, so large M may return FA_ERR_ARG). */
fa_status fa_search(fa_index *ix, const float *queries, int64_t nq, int32_t d, int32_t k,
                    int32_t nprobe, int64_t *out_ids, float *out_dist);

/* Top-k search with explicit parameters (precision, re-rank, per-query k and
 * nprobe, device-resident buffers, stream). With FA_QUERIES_ON_DEVICE /
 * FA_OUTPUTS_ON_DEVICE the pointers are device pointers on the index's device;
 * otherwise host pointers (pinned memory gives overlapped copies). */
fa_status fa_search_ex(fa_index *ix, const float *queries, int64_t nq, int32_t d, int32_t k,
                       int32_t nprobe, const fa_search_params *sp, int64_t *out_ids,
                       float *out_dist);

/* Autotuning of the scan launch (the batching form's tile shape). */
typedef struct fa_tune_result {
    int32_t variants, chosen;         /* variants timed; index of the fastest */
    int32_t threads[8], ilp[8], persistent[8];
    int32_t tile_chunks[8];           /* > 0: tiled form, 32-candidate chunks per tile */
    float ms[8];                      /* median device time of the scan stage */
} fa_tune_result;

/* Times the launch shapes of the ADC scan on the given host queries with the
 * given parameters and keeps the fastest in the index for later calls of the
 * same class (top-n above or below 256, LUT in the scan CTA or in HBM):
 *   - one CTA per query: 256 or 512 threads per CTA, one or two 32-candidate
 *     chunks in flight per warp;
 *   - the tiled batching form: persistent CTAs pull tiles of T chunks of one
 *     query (T = 64, 256, 1024), each tile's top-n is merged per query.
 * Every variant must return the same rows bit for bit (else FA_ERR_STATE).
 * Calls made before tuning use 256 threads, one chunk, one CTA per query;
 * FA_PERSISTENT selects the tiled form with T = 256 unless tuned. */
fa_status fa_autotune(fa_index *ix, const float *queries, int64_t nq, int32_t d, int32_t k,
                      int32_t nprobe, const fa_search_params *sp, fa_tune_result *out);

/* ------------------------------------------------------------------------- */
/* Serving form: continuous batching of single-query requests                */
/* ------------------------------------------------------------------------- */

typedef struct fa_server fa_server; /* opaque, owned by the library */

typedef struct fa_server_params {
    int32_t max_batch;        /* requests per batch at most */
    int32_t window_us;        /* a batch closes when its oldest request waited this long */
    int32_t slots;            /* batches in flight at most (device memory blocks) */
    int32_t kmax;             /* largest k a request may ask for (<= 256) */
    int32_t nprobe_max;       /* larger per-request nprobe values are clamped to this */
    int32_t pad0;
    int64_t mem_budget_bytes; /* > 0: cap on the slots' device memory (fewer slots) */
} fa_server_params;

typedef struct fa_server_stats_t {
    int64_t batches, requests, pending, device_bytes;
    int32_t inflight_batches, slots;
} fa_server_stats_t;

/* Defaults: batches of up to 1024 requests, 200 us window, 4 slots, kmax 100,
 * nprobe_max 256, no memory cap. */
void fa_server_params_init(fa_server_params *p);

/* Starts a request loop over ix with the search parameters sp (precision,
 * re-rank, ...; buffer flags and per-query pointers are set by the loop, and
 * batches always run the tiled persistent scan of FA_PERSISTENT). The
 * loop (a host thread) closes a batch when it is full or its oldest request
 * has waited window_us, admits it when one of the `slots` device memory blocks
 * is free (blocks are allocated here, none in the loop), and launches it
 * without waiting, so batches overlap on the device. The paper runs one CPU
 * thread per query against a pool of per-query GPU blocks (§5); here requests
 * share batches and a block serves one batch. */
fa_status fa_server_create(fa_index *ix, const fa_server_params *p, const fa_search_params *sp,
                           fa_server **out);

/* Queues n requests: queries[n][d] (host), k[n] in 1..kmax, nprobe[n] >= 1.
 * out_request_ids (optional) receives each request's id. */
fa_status fa_server_submit(fa_server *sv, const float *queries, int64_t n, const int32_t *k,
                           const int32_t *nprobe, int64_t *out_request_ids);

/* Takes up to max_results completed requests (waits up to timeout_us for the
 * first): request id, ids and distances [max_results][kstride] (padded with
 * -1 / +inf past each request's k), latency from submit to completion in us,
 * and status. Returns how many were written. */
int64_t fa_server_poll(fa_server *sv, int64_t max_results, int32_t timeout_us, int64_t *request_ids,
                       int64_t *ids, float *dist, int32_t kstride, double *latency_us,
                       int32_t *status);

fa_status fa_server_stats(fa_server *sv, fa_server_stats_t *out);

/* Finishes every queued request, then stops the loop and frees its memory. */
void fa_server_destroy(fa_server *sv);

/* ------------------------------------------------------------------------- */
/* Test hooks (host buffers)                                                 */
/* ------------------------------------------------------------------------- */

/* Coarse probe (step 2) only: out_probes[nq][nprobe] ascending by distance. */
fa_status fa_debug_probes(fa_index *ix, const float *queries, int64_t nq, int32_t nprobe,
                          const fa_search_params *sp, int32_t *out_probes);

/* Gather + dedup (steps 3-5) of one query as run on the GPU: the distinct
 * vector ids of the probed lists, ascending. probes[nprobe] gives the lists
 * (NULL runs the coarse probe). *out_n receives the count; FA_ERR_OVERFLOW
 * if it exceeds cap. */
fa_status fa_debug_candidates(fa_index *ix, const float *query, int32_t nprobe,
                              const int32_t *probes, int64_t *out_ids, int64_t cap,
                              int64_t *out_n);

/* The lookup table of one query (step 1) as the scan reads it, dequantized to
 * float: out_lut[M][256]. */
fa_status fa_debug_lut(fa_index *ix, const float *query, const fa_search_params *sp,
                       float *out_lut);

/* Failure injection on the host (no counterpart in the paper): the n-th next
 * device allocation of the library (index upload, workspaces, server slots)
 * fails as if the device were out of memory; the call returns FA_ERR_OOM and
 * leaves the index usable. n = 0 turns it off. */
fa_status fa_debug_fail_alloc(int32_t n);

/* Runs one device wait that must run out: a CTA waits, with the library's
 * bounded mbarrier wait, for a phase nothing completes and polls a flag
 * nothing sets, `polls` tries each. Returns FA_ERR_TIMEOUT from the device
 * status word; the CUDA context stays usable. FA_ERR_NODEV without a GPU. */
fa_status fa_debug_timeout(uint32_t polls);

/* Builds the navigation graph of the index's lists (§4.1 "In-memory
 * Indices") for FA_PROBE_GRAPH, replacing any earlier one. Vertex v is list
 * v with a head vector: its centroid, rounded to the nearest integer (halves
 * to even) and clipped to the type's range for uint8 / int8 vectors. Out-edges
 * of vertex u (squared L2 between heads, ties by id; its K = 3R nearest
 * other vertices found exactly on the GPU are the candidates): the
 * candidates kept by relative-neighbourhood pruning (in distance order, one
 * is dropped when an already kept one is strictly closer to it than u is;
 * SPTAG prunes its graph this way); then the vertices that kept u, nearest
 * first (the neighbours' update when the paper inserts a vertex); then
 * u's nearest candidates, up to R edges. S pivot
 * vertices i * nlist / S are the walks' seeds: each walk starts from the
 * pivots nearest its query (graph_entry). R in 1..64 (0: 32), S in
 * 1..4096 (0: min(4096, max(64, nlist / 64))), both capped by nlist. The
 * graph is not saved with the index. FA_ERR_ARG on bad sizes. */
fa_status fa_build_probe_graph(fa_index *ix, int32_t R, int32_t S);

/* Copies the navigation graph out: adj [nlist][R] (-1 = no edge) and seeds
 * [S] (either may be NULL), *R and *S. FA_ERR_ARG when there is none. */
fa_status fa_index_get_graph(fa_index *ix, int32_t *adj, int32_t *seeds, int32_t *R, int32_t *S);

/* The graph walk alone for host queries [nq][d]: probes [nq][nprobe] (-1
 * past the lists found), found [nq] lists found, checks [nq] vertices
 * checked (either may be NULL). beam, max_check and entry as in
 * fa_search_params (0 = their defaults). */
fa_status fa_debug_graph_probe(fa_index *ix, const float *queries, int64_t nq, int32_t nprobe,
                               int32_t beam, int32_t max_check, int32_t entry, int32_t *probes,
                               int32_t *found, int32_t *checks);

/* The storage layout of FA_RAW_HOST_PAGED raw vectors (§4.3): page_of[v]
 * and slot_of[v] (host [n], caller ids) receive each vector's page and its
 * row in that page; *rows_per_page and *pages the page capacity and count.
 * FA_ERR_ARG when the index's raw vectors are not paged. */
fa_status fa_debug_page_map(fa_index *ix, int64_t *page_of, int32_t *slot_of, int32_t *rows_per_page,
                            int64_t *pages);

/* Sets how many standard deviations above the expected count the scan's
 * sampled threshold estimate sits (a top-n above 256 over many more
 * candidates first scores a strided sample of them; default 4). The estimate
 * is only a filter: when fewer than n keys fall below it the query is scanned
 * again without it, and when more fall below it than shared memory holds the
 * query is scanned again with the threshold tightening as it goes, so results
 * do not depend on sigma. A large negative or positive sigma forces those
 * second scans, which is how tests reach them.
 * Process-wide; not thread-safe against concurrent searches. */
fa_status fa_debug_tau_sigma(float sigma);

/* ------------------------------------------------------------------------- */
/* Coarse probe without allocation                                           */
/* ------------------------------------------------------------------------- */

/* The coarse probe (step 2) for callers that cannot allocate device memory
 * (the paper has no counterpart; it is an addition of this library). Such
 * callers are processes whose device memory is owned in full by another
 * allocator or a fixed budget, and latency-bound code that cannot afford the
 * synchronisation and unbounded time of a cudaMalloc in the middle of its work.
 *
 * queries[nq][d] and centroids[nlist][d] are float32 device pointers on the
 * current device (make the device that owns the buffers current first);
 * probes[nq][nprobe] (int32, device) receives each query's nprobe nearest
 * centroids by squared L2, ascending by (distance, centroid index), computed
 * by the same kernels as the coarse probe of fa_search. The work is enqueued
 * on `stream` (a cudaStream_t, NULL = legacy default stream); results are
 * ready when the stream is.
 *
 * Scratch: a 16 MiB array in this library's device image (4194304 float
 * distances), held by every GPU that loads the library until the process
 * exits. No cudaMalloc, cudaFree or allocating library routine is called. The
 * first call on each device looks the array's device address up (once, with
 * that device current); make that first call before any stream capture.
 * Every call shares the array and overwrites what it reads, so calls that
 * overlap on the GPU race: serialise them.
 *
 * Errors: FA_ERR_ARG for nq < 0, d < 1, nprobe outside 1..min(nlist, 512),
 * null buffers, or nlist above 4194304 (the scratch capacity); FA_ERR_CUDA if
 * a launch fails. nq == 0 returns FA_OK without touching the GPU. */
fa_status fa_coarse_probe_noalloc(const float *queries, int64_t nq, int32_t d,
                                  const float *centroids, int32_t nlist, int32_t nprobe,
                                  int32_t *probes, void *stream);

/* ------------------------------------------------------------------------- */
/* Errors and version                                                        */
/* ------------------------------------------------------------------------- */

const char *fa_last_error(void);          /* message of this thread's last failure */
const char *fa_status_str(fa_status s);   /* static name of a status */
const char *fa_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FA_H */
