/*
 * FP64 CPU oracle for the IVF-PQ filtering path of FusionANNS (arXiv 2409.16576).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU
 * baseline leg may load this library. It shares no code, header, table or
 * helper with the CUDA path, and the CUDA path never calls it.
 *
 * It works on the *logical* index: each posting list is a plain array of
 * vector ids (the paper's list metadata, §4.1 "In-memory Indices"), PQ codes
 * are an [n][M] byte matrix indexed by vector id (§4.1 "PQ-based Vectors in
 * GPU's HBM"), and the M sub-codebooks hold 256 centroids of d/M dimensions
 * each (§2.2). Every step below follows the online processing order of §3
 * (steps 1-8) and is written as its plain definition in double precision:
 *
 *   coarse probe   the m = nprobe lists whose centroids are nearest to q
 *                  (step 2; exact top-m), or the paper's walk over a
 *                  navigation graph of the lists (§4.1 "In-memory Indices")
 *   gather         the ids of the probed lists (steps 3-4)
 *   dedup          the set of distinct ids, emitted sorted ascending (step 5)
 *   LUT            dist(q_i, c) for every subspace i and centroid c (step 1)
 *   ADC            Eq. 1: sum over the M subspaces of LUT[i][code_i(v)] (step 6)
 *   top-n          the n smallest (distance, id) pairs, ascending (step 7)
 *   re-rank        Algorithm 1 with the change rate of Eq. 3 (step 8, §4.2)
 *
 * Readings of points the paper leaves open (all used consistently here):
 *   - dist() in Eq. 1 is the squared L2 distance; it is the form that splits
 *     into a sum over subspaces.
 *   - subspaces are contiguous blocks of dsub = d / M coordinates (§2.2
 *     "divided evenly").
 *   - ties are broken by the smaller vector (or list) id everywhere.
 *   - a heap insertion needs (dist, id) strictly below the heap maximum
 *     (§4.2, "less than the current maximum"); while the heap holds fewer
 *     than k entries every candidate is inserted.
 *   - the stop test is the one Algorithm 1 writes: Delta <= eps increments
 *     the stability counter and counter >= beta ends the loop; a ragged last
 *     mini-batch stops at the end of the task list.
 *   - Delta keeps k as its denominator even while the heap holds fewer than k.
 *   - rows with fewer than k results are padded with (id -1, +inf).
 *   - inner-product search (the second metric of the SPACEV-like workload,
 *     Table 1) ranks by the smallest -<q, x>: the coarse probe by -<q, c>,
 *     the table entries are -<q_i, C_i[c]> (which Eq. 1 adds up like the L2
 *     terms, since the inner product also splits over subspaces), and the
 *     re-rank and the ground truth use the exact -<q, x>.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_RAW_U8 1
#define OR_RAW_F32 0
#define OR_RAW_I8 2

#define OR_L2 0
#define OR_IP 1

typedef struct {
    double d;
    int64_t id;
} pair_t;

static int pair_less(const pair_t *a, const pair_t *b)
{
    if (a->d < b->d) return 1;
    if (a->d > b->d) return 0;
    return a->id < b->id;
}

static int pair_cmp(const void *pa, const void *pb)
{
    const pair_t *a = (const pair_t *)pa, *b = (const pair_t *)pb;
    if (pair_less(a, b)) return -1;
    if (pair_less(b, a)) return 1;
    return 0;
}

static int u32_cmp(const void *pa, const void *pb)
{
    uint32_t a = *(const uint32_t *)pa, b = *(const uint32_t *)pb;
    return (a > b) - (a < b);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ---------------------------------------------------------------------------
 * Step 2 (coarse probe): squared L2 from q to every list centroid, in FP64,
 * and the nprobe smallest by (distance, list id).
 * ------------------------------------------------------------------------- */
static void coarse_one(const float *q, int32_t d, const float *cent, int32_t nlist,
                       int32_t nprobe, int32_t *probes, double *d2out, pair_t *scratch,
                       int32_t metric)
{
    for (int32_t l = 0; l < nlist; ++l) {
        double s = 0.0;
        const float *c = cent + (int64_t)l * d;
        if (metric == OR_IP) {
            for (int32_t j = 0; j < d; ++j) s -= (double)q[j] * (double)c[j];
        } else {
            for (int32_t j = 0; j < d; ++j) {
                double t = (double)q[j] - (double)c[j];
                s += t * t;
            }
        }
        scratch[l].d = s;
        scratch[l].id = l;
    }
    qsort(scratch, (size_t)nlist, sizeof(pair_t), pair_cmp);
    for (int32_t i = 0; i < nprobe; ++i) {
        probes[i] = (int32_t)scratch[i].id;
        if (d2out) d2out[i] = scratch[i].d;
    }
}

void or_coarse_m(const float *q, int64_t nq, int32_t d, const float *cent, int32_t nlist,
                 int32_t nprobe, int32_t *probes, double *d2out, int32_t metric)
{
#pragma omp parallel
    {
        pair_t *scratch = (pair_t *)malloc(sizeof(pair_t) * (size_t)nlist);
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < nq; ++i)
            coarse_one(q + i * d, d, cent, nlist, nprobe, probes + i * nprobe,
                       d2out ? d2out + i * nprobe : NULL, scratch, metric);
        free(scratch);
    }
}

void or_coarse(const float *q, int64_t nq, int32_t d, const float *cent, int32_t nlist,
               int32_t nprobe, int32_t *probes, double *d2out)
{
    or_coarse_m(q, nq, d, cent, nlist, nprobe, probes, d2out, OR_L2);
}

/* ---------------------------------------------------------------------------
 * Step 1 (distance table): LUT[i][c] = sum over the coordinates j of subspace
 * i of (q_j - C_i[c][j])^2, the dist(q_i, c_i) terms that Eq. 1 adds up.
 * codebooks is [M][256][dsub]; lut is [M][256].
 * ------------------------------------------------------------------------- */
void or_lut_m(const float *q, int32_t d, int32_t M, const float *codebooks, double *lut,
              int32_t metric)
{
    int32_t dsub = d / M;
    for (int32_t i = 0; i < M; ++i)
        for (int32_t c = 0; c < 256; ++c) {
            const float *cw = codebooks + ((int64_t)i * 256 + c) * dsub;
            double s = 0.0;
            if (metric == OR_IP) {
                for (int32_t j = 0; j < dsub; ++j) s -= (double)q[i * dsub + j] * (double)cw[j];
            } else {
                for (int32_t j = 0; j < dsub; ++j) {
                    double t = (double)q[i * dsub + j] - (double)cw[j];
                    s += t * t;
                }
            }
            lut[i * 256 + c] = s;
        }
}

void or_lut(const float *q, int32_t d, int32_t M, const float *codebooks, double *lut)
{
    or_lut_m(q, d, M, codebooks, lut, OR_L2);
}

/* ---------------------------------------------------------------------------
 * Steps 3-5 (gather, dedup): concatenate the id arrays of the probed lists,
 * then sort and keep each distinct id once. Returns the number of distinct
 * ids (written ascending to out, which must hold the gathered count);
 * *gathered receives the size of the concatenation.
 * ------------------------------------------------------------------------- */
int64_t or_candidates(const int32_t *probes, int32_t nprobe, const int64_t *list_off,
                      const int64_t *list_ids, uint32_t *out, int64_t cap, int64_t *gathered)
{
    int64_t g = 0;
    for (int32_t p = 0; p < nprobe; ++p) {
        int32_t l = probes[p];
        for (int64_t e = list_off[l]; e < list_off[l + 1]; ++e) {
            if (g < cap) out[g] = (uint32_t)list_ids[e];
            ++g;
        }
    }
    if (gathered) *gathered = g;
    if (g > cap) return -1;
    qsort(out, (size_t)g, sizeof(uint32_t), u32_cmp);
    int64_t u = 0;
    for (int64_t i = 0; i < g; ++i)
        if (u == 0 || out[i] != out[u - 1]) out[u++] = out[i];
    return u;
}

/* Step 6, Eq. 1: ADC distance of vector v = sum_i LUT[i][code[v][i]]. */
void or_adc(const double *lut, int32_t M, const uint8_t *codes, const uint32_t *ids,
            int64_t n, double *dist)
{
    for (int64_t t = 0; t < n; ++t) {
        const uint8_t *cv = codes + (int64_t)ids[t] * M;
        double s = 0.0;
        for (int32_t i = 0; i < M; ++i) s += lut[i * 256 + cv[i]];
        dist[t] = s;
    }
}

/* Step 7: the n smallest (dist, id) pairs in ascending order; rows shorter
 * than n are padded with (-1, +inf). */
void or_topn(const double *dist, const uint32_t *ids, int64_t cnt, int32_t n,
             int64_t *out_ids, double *out_dist)
{
    pair_t *p = (pair_t *)malloc(sizeof(pair_t) * (size_t)(cnt > 0 ? cnt : 1));
    for (int64_t i = 0; i < cnt; ++i) {
        p[i].d = dist[i];
        p[i].id = ids[i];
    }
    qsort(p, (size_t)cnt, sizeof(pair_t), pair_cmp);
    for (int32_t i = 0; i < n; ++i) {
        if (i < cnt) {
            out_ids[i] = p[i].id;
            out_dist[i] = p[i].d;
        } else {
            out_ids[i] = -1;
            out_dist[i] = INFINITY;
        }
    }
    free(p);
}

/* Coordinate j of raw vector v (uint8, int8 or float32 rows). */
static double raw_at(const void *raw, int32_t raw_dtype, int32_t d, int64_t v, int32_t j)
{
    if (raw_dtype == OR_RAW_U8) return (double)((const uint8_t *)raw)[v * d + j];
    if (raw_dtype == OR_RAW_I8) return (double)((const int8_t *)raw)[v * d + j];
    return (double)((const float *)raw)[v * d + j];
}

/* Exact distance between q and raw vector v: squared L2, or -<q, x>. */
static double exact_dist(const float *q, int32_t d, const void *raw, int32_t raw_dtype, int64_t v,
                         int32_t metric)
{
    double s = 0.0;
    for (int32_t j = 0; j < d; ++j) {
        const double x = raw_at(raw, raw_dtype, d, v, j);
        if (metric == OR_IP) {
            s -= (double)q[j] * x;
        } else {
            double t = (double)q[j] - x;
            s += t * t;
        }
    }
    return s;
}

void or_exact_m(const float *q, int32_t d, const void *raw, int32_t raw_dtype,
                const int64_t *ids, int64_t n, double *out, int32_t metric)
{
    for (int64_t i = 0; i < n; ++i) out[i] = exact_dist(q, d, raw, raw_dtype, ids[i], metric);
}

void or_exact_l2(const float *q, int32_t d, const void *raw, int32_t raw_dtype,
                 const int64_t *ids, int64_t n, double *out)
{
    or_exact_m(q, d, raw, raw_dtype, ids, n, out, OR_L2);
}

/* ---------------------------------------------------------------------------
 * Step 8, Algorithm 1 (heuristic re-ranking) with Eq. 3. The max-heap Q is
 * kept as a small array sorted ascending; its last element is the maximum.
 * tasks: candidate ids in ascending ADC order (entries < 0 are skipped as
 * padding). Returns the number of mini-batches processed.
 * ------------------------------------------------------------------------- */
static int in_set(const int64_t *s, int32_t n, int64_t id)
{
    for (int32_t i = 0; i < n; ++i)
        if (s[i] == id) return 1;
    return 0;
}

int32_t or_rerank_m(const float *q, int32_t d, const void *raw, int32_t raw_dtype,
                    const int64_t *tasks, int32_t ntasks, int32_t k, int32_t batch,
                    float eps, int32_t beta, int64_t *out_ids, double *out_dist, int32_t metric)
{
    pair_t *Q = (pair_t *)malloc(sizeof(pair_t) * (size_t)(k + 1));
    int64_t *prev = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    int32_t qn = 0, counter = 0, batches = 0;
    int32_t valid = 0;
    while (valid < ntasks && tasks[valid] >= 0) ++valid;

    for (int32_t i = 0; i < valid; i += batch) {
        /* S_{n-1} <- ids currently in Q */
        int32_t pn = qn;
        for (int32_t t = 0; t < qn; ++t) prev[t] = Q[t].id;
        int32_t end = i + batch < valid ? i + batch : valid;
        for (int32_t j = i; j < end; ++j) {
            pair_t c;
            c.id = tasks[j];
            c.d = exact_dist(q, d, raw, raw_dtype, tasks[j], metric);
            if (qn < k || pair_less(&c, &Q[qn - 1])) {
                /* insert in order, drop the maximum when over k */
                int32_t pos = qn < k ? qn : k - 1;
                if (qn < k) ++qn;
                while (pos > 0 && pair_less(&c, &Q[pos - 1])) {
                    Q[pos] = Q[pos - 1];
                    --pos;
                }
                Q[pos] = c;
            }
        }
        ++batches;
        /* Eq. 3: Delta = |S_n - S_n intersect S_{n-1}| / k */
        int32_t changed = 0;
        for (int32_t t = 0; t < qn; ++t)
            if (!in_set(prev, pn, Q[t].id)) ++changed;
        double delta = (double)changed / (double)k;
        if (delta <= (double)eps) {
            ++counter;
            if (counter >= beta) break;
        } else {
            counter = 0;
        }
    }
    for (int32_t t = 0; t < k; ++t) {
        if (t < qn) {
            out_ids[t] = Q[t].id;
            out_dist[t] = Q[t].d;
        } else {
            out_ids[t] = -1;
            out_dist[t] = INFINITY;
        }
    }
    free(Q);
    free(prev);
    return batches;
}

int32_t or_rerank(const float *q, int32_t d, const void *raw, int32_t raw_dtype,
                  const int64_t *tasks, int32_t ntasks, int32_t k, int32_t batch,
                  float eps, int32_t beta, int64_t *out_ids, double *out_dist)
{
    return or_rerank_m(q, d, raw, raw_dtype, tasks, ntasks, k, batch, eps, beta, out_ids,
                       out_dist, OR_L2);
}

/* ---------------------------------------------------------------------------
 * The whole filtering path for nq queries (steps 1-8 of §3), one query per
 * OpenMP iteration.
 *
 *   probes_in  optional [nq][nprobe] probe lists; NULL runs the coarse probe.
 *   rerank_n   0: return the ADC top-k. >0: take the ADC top-rerank_n and
 *              re-rank them with Algorithm 1 (needs raw vectors).
 *   stats      optional [nq][4]: gathered ids, distinct ids, mini-batches run,
 *              candidates handed to the re-rank.
 * ------------------------------------------------------------------------- */
int32_t or_search_m(const float *queries, int64_t nq, int32_t d, const float *cent, int32_t nlist,
                    int32_t M, const float *codebooks, const uint8_t *codes, const int64_t *list_off,
                    const int64_t *list_ids, const void *raw, int32_t raw_dtype, int32_t nprobe,
                    int32_t k, const int32_t *probes_in, int32_t rerank_n, int32_t batch, float eps,
                    int32_t beta, int64_t *out_ids, double *out_dist, int64_t *stats, int32_t metric)
{
    if (nprobe > nlist) nprobe = nlist;
    if (nprobe < 1) nprobe = 1;
    int64_t maxlist = 0;
    for (int32_t l = 0; l < nlist; ++l)
        if (list_off[l + 1] - list_off[l] > maxlist) maxlist = list_off[l + 1] - list_off[l];
    int64_t cap = maxlist * nprobe;
    int32_t n_top = rerank_n > 0 ? rerank_n : k;
    int32_t err = 0;

#pragma omp parallel
    {
        pair_t *scratch = (pair_t *)malloc(sizeof(pair_t) * (size_t)nlist);
        int32_t *probes = (int32_t *)malloc(sizeof(int32_t) * (size_t)nprobe);
        uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(cap > 0 ? cap : 1));
        double *dist = (double *)malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
        double *lut = (double *)malloc(sizeof(double) * (size_t)M * 256);
        int64_t *top_ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_top);
        double *top_d = (double *)malloc(sizeof(double) * (size_t)n_top);
#pragma omp for schedule(dynamic, 1)
        for (int64_t qi = 0; qi < nq; ++qi) {
            const float *q = queries + qi * d;
            if (probes_in)
                memcpy(probes, probes_in + qi * nprobe, sizeof(int32_t) * (size_t)nprobe);
            else
                coarse_one(q, d, cent, nlist, nprobe, probes, NULL, scratch, metric);
            or_lut_m(q, d, M, codebooks, lut, metric);
            int64_t gathered = 0;
            int64_t u = or_candidates(probes, nprobe, list_off, list_ids, cand, cap, &gathered);
            if (u < 0) {
                err = 1;
                continue;
            }
            or_adc(lut, M, codes, cand, u, dist);
            or_topn(dist, cand, u, n_top, top_ids, top_d);
            int32_t batches = 0;
            if (rerank_n > 0) {
                batches = or_rerank_m(q, d, raw, raw_dtype, top_ids, n_top, k, batch, eps, beta,
                                      out_ids + qi * k, out_dist + qi * k, metric);
            } else {
                memcpy(out_ids + qi * k, top_ids, sizeof(int64_t) * (size_t)k);
                memcpy(out_dist + qi * k, top_d, sizeof(double) * (size_t)k);
            }
            if (stats) {
                stats[qi * 4 + 0] = gathered;
                stats[qi * 4 + 1] = u;
                stats[qi * 4 + 2] = batches;
                stats[qi * 4 + 3] = u < n_top ? u : n_top;
            }
        }
        free(scratch);
        free(probes);
        free(cand);
        free(dist);
        free(lut);
        free(top_ids);
        free(top_d);
    }
    return err ? -1 : 0;
}

int32_t or_search(const float *queries, int64_t nq, int32_t d, const float *cent, int32_t nlist,
                  int32_t M, const float *codebooks, const uint8_t *codes, const int64_t *list_off,
                  const int64_t *list_ids, const void *raw, int32_t raw_dtype, int32_t nprobe,
                  int32_t k, const int32_t *probes_in, int32_t rerank_n, int32_t batch, float eps,
                  int32_t beta, int64_t *out_ids, double *out_dist, int64_t *stats)
{
    return or_search_m(queries, nq, d, cent, nlist, M, codebooks, codes, list_off, list_ids, raw,
                       raw_dtype, nprobe, k, probes_in, rerank_n, batch, eps, beta, out_ids, out_dist,
                       stats, OR_L2);
}

/* ---------------------------------------------------------------------------
 * Ground truth: brute-force k nearest neighbours by exact squared L2 in FP64
 * (exact for uint8 data), ties by smaller id. Used for Recall@k (§6).
 * ------------------------------------------------------------------------- */
void or_knn_m(const float *queries, int64_t nq, const void *base, int32_t raw_dtype, int64_t n,
              int32_t d, int32_t k, int64_t *out_ids, double *out_dist, int32_t metric)
{
#pragma omp parallel
    {
        pair_t *Q = (pair_t *)malloc(sizeof(pair_t) * (size_t)(k + 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t qi = 0; qi < nq; ++qi) {
            const float *q = queries + qi * d;
            int32_t qn = 0;
            for (int64_t v = 0; v < n; ++v) {
                pair_t c;
                c.id = v;
                c.d = exact_dist(q, d, base, raw_dtype, v, metric);
                if (qn < k || pair_less(&c, &Q[qn - 1])) {
                    int32_t pos = qn < k ? qn : k - 1;
                    if (qn < k) ++qn;
                    while (pos > 0 && pair_less(&c, &Q[pos - 1])) {
                        Q[pos] = Q[pos - 1];
                        --pos;
                    }
                    Q[pos] = c;
                }
            }
            for (int32_t t = 0; t < k; ++t) {
                out_ids[qi * k + t] = t < qn ? Q[t].id : -1;
                out_dist[qi * k + t] = t < qn ? Q[t].d : INFINITY;
            }
        }
        free(Q);
    }
}

void or_knn(const float *queries, int64_t nq, const void *base, int32_t raw_dtype, int64_t n,
            int32_t d, int32_t k, int64_t *out_ids, double *out_dist)
{
    or_knn_m(queries, nq, base, raw_dtype, n, d, k, out_ids, out_dist, OR_L2);
}

/* ---------------------------------------------------------------------------
 * Redundancy-aware I/O deduplication (§4.3).
 *
 * Storage layout: list l's bucket holds the raw vectors whose primary list is
 * l (a vector is stored once, in one bucket), in ascending id order. A page
 * holds cap vectors. Each bucket first fills whole pages of its own; the
 * rest of it (its unaligned portion, 0 < size < cap) is a tail, and tails are
 * combined into shared pages by a max-min rule: the largest tail not yet
 * placed opens a page, then the smallest remaining tails join it in
 * ascending size while they fit; ties by list id. Pages are numbered in the
 * order they are created: every bucket's whole pages first (by list id),
 * then the shared pages. page_of[v] and slot_of[v] give a vector's page and
 * position in it. Returns the number of pages.
 * ------------------------------------------------------------------------- */
typedef struct {
    int64_t size;
    int32_t list;
} tail_t;

static int tail_desc(const void *pa, const void *pb)
{
    const tail_t *a = (const tail_t *)pa, *b = (const tail_t *)pb;
    if (a->size != b->size) return a->size > b->size ? -1 : 1;
    return (a->list > b->list) - (a->list < b->list);
}

int64_t or_page_layout(const int32_t *primary, int64_t n, int32_t nlist, int32_t cap,
                       int64_t *page_of, int32_t *slot_of)
{
    int64_t *cnt = (int64_t *)calloc((size_t)nlist + 1, sizeof(int64_t));
    for (int64_t v = 0; v < n; ++v) cnt[primary[v] + 1]++;
    for (int32_t l = 0; l < nlist; ++l) cnt[l + 1] += cnt[l];
    int64_t *mem = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nlist);
    for (int32_t l = 0; l < nlist; ++l) fill[l] = cnt[l];
    for (int64_t v = 0; v < n; ++v) mem[fill[primary[v]]++] = v; /* ascending ids per bucket */
    int64_t page = 0;
    tail_t *tails = (tail_t *)malloc(sizeof(tail_t) * (size_t)(nlist > 0 ? nlist : 1));
    int32_t nt = 0;
    for (int32_t l = 0; l < nlist; ++l) {
        const int64_t b = cnt[l], e = cnt[l + 1], whole = (e - b) / cap;
        for (int64_t t = 0; t < whole * cap; ++t) {
            page_of[mem[b + t]] = page + t / cap;
            slot_of[mem[b + t]] = (int32_t)(t % cap);
        }
        page += whole;
        if ((e - b) % cap) {
            tails[nt].size = (e - b) % cap;
            tails[nt].list = l;
            ++nt;
        }
    }
    qsort(tails, (size_t)nt, sizeof(tail_t), tail_desc);
    char *used = (char *)calloc((size_t)(nt > 0 ? nt : 1), 1);
    int32_t hi = 0, lo = nt - 1; /* largest and smallest unplaced tails */
    while (hi <= lo) {
        if (used[hi]) { ++hi; continue; }
        int64_t room = cap, slot = 0;
        int32_t pick = hi;
        for (;;) {
            const int32_t l = tails[pick].list;
            const int64_t b = cnt[l + 1] - tails[pick].size;
            for (int64_t t = 0; t < tails[pick].size; ++t) {
                page_of[mem[b + t]] = page;
                slot_of[mem[b + t]] = (int32_t)(slot + t);
            }
            slot += tails[pick].size;
            room -= tails[pick].size;
            used[pick] = 1;
            while (lo > hi && used[lo]) --lo;
            if (lo <= hi || tails[lo].size > room) break;
            pick = lo;
        }
        ++page;
        ++hi;
    }
    free(used);
    free(tails);
    free(fill);
    free(mem);
    free(cnt);
    return page;
}

/* Algorithm 1 (as or_rerank_m) counting page reads: each mini-batch reads
 * the distinct pages of its tasks once (intra-mini-batch merge), except pages
 * the query read in an earlier mini-batch, which its buffer holds
 * (inter-mini-batch deduplication); *pages_read receives the total. */
int32_t or_rerank_pages(const float *q, int32_t d, const void *raw, int32_t raw_dtype,
                        const int64_t *tasks, int32_t ntasks, int32_t k, int32_t batch, float eps,
                        int32_t beta, const int64_t *page_of, int64_t *out_ids, double *out_dist,
                        int32_t metric, int64_t *pages_read)
{
    int32_t valid = 0;
    while (valid < ntasks && tasks[valid] >= 0) ++valid;
    int32_t nb = or_rerank_m(q, d, raw, raw_dtype, tasks, ntasks, k, batch, eps, beta, out_ids,
                             out_dist, metric);
    int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(valid > 0 ? valid : 1));
    int64_t nbuf = 0, reads = 0;
    for (int32_t b = 0; b < nb; ++b) {
        const int32_t i0 = b * batch, i1 = i0 + batch < valid ? i0 + batch : valid;
        for (int32_t j = i0; j < i1; ++j) {
            const int64_t pg = page_of[tasks[j]];
            int seen = 0;
            for (int64_t t = 0; t < nbuf; ++t)
                if (buf[t] == pg) { seen = 1; break; }
            if (!seen) {
                buf[nbuf++] = pg;
                ++reads;
            }
        }
    }
    free(buf);
    *pages_read = reads;
    return nb;
}


/* ---------------------------------------------------------------------------
 * Step 2 by the navigation graph (§3 step 2, §4.1 "In-memory Indices"): the
 * vertices are the lists, each with a vertex vector (its head), and each
 * vertex has up to R out-edges (adj[v][0..R), -1 = none). A query walks the
 * graph best first:
 *   - every seed is evaluated first (a seed already seen is skipped);
 *   - evaluating a vertex marks it seen, counts one check and offers it to
 *     the beam, the L best (distance, id) pairs seen so far: it enters when
 *     the beam holds fewer than L or it is below the beam's last pair;
 *   - then, while fewer than max_check vertices were checked and the beam
 *     holds a vertex not yet expanded, the first such vertex (in beam order)
 *     is expanded: each of its out-neighbours not yet seen is evaluated, in
 *     the order of its edge list;
 *   - the top-m lists are the first min(m, beam size) pairs of the beam.
 * Returns how many lists were written to out. Distances are squared L2 (or
 * -<q, h> with metric IP) in FP64 against the heads.
 * ------------------------------------------------------------------------- */
static void beam_offer(pair_t *beam, int32_t *bn, int32_t L, double dv, int64_t v)
{
    pair_t x = {dv, v};
    if (*bn == L && !pair_less(&x, &beam[L - 1])) return;
    int32_t i = *bn < L ? *bn : L - 1;  /* slot freed at the end */
    while (i > 0 && pair_less(&x, &beam[i - 1])) {
        beam[i] = beam[i - 1];
        --i;
    }
    beam[i] = x;
    if (*bn < L) ++*bn;
}

static double head_dist(const float *q, const double *h, int32_t d, int32_t metric)
{
    double s = 0.0;
    for (int32_t j = 0; j < d; ++j) {
        if (metric == OR_IP) {
            s -= (double)q[j] * h[j];
        } else {
            double t = (double)q[j] - h[j];
            s += t * t;
        }
    }
    return s;
}

int32_t or_graph_walk(const float *q, int32_t d, const double *heads, int32_t nlist,
                      const int32_t *adj, int32_t R, const int32_t *seeds, int32_t S, int32_t L,
                      int32_t max_check, int32_t nprobe, int32_t metric, int32_t *out,
                      int32_t *checks_out)
{
    char *seen = (char *)calloc((size_t)nlist, 1);
    char *expanded = (char *)calloc((size_t)nlist, 1);
    pair_t *beam = (pair_t *)malloc(sizeof(pair_t) * (size_t)L);
    int32_t bn = 0, checks = 0;
    for (int32_t s = 0; s < S; ++s) {
        int32_t v = seeds[s];
        if (seen[v]) continue;
        seen[v] = 1;
        ++checks;
        beam_offer(beam, &bn, L, head_dist(q, heads + (int64_t)v * d, d, metric), v);
    }
    while (checks < max_check) {
        int32_t i = 0;
        while (i < bn && expanded[beam[i].id]) ++i;
        if (i == bn) break;  /* every vertex of the beam is expanded */
        int64_t p = beam[i].id;
        expanded[p] = 1;
        for (int32_t e = 0; e < R; ++e) {
            int32_t u = adj[p * R + e];
            if (u < 0 || seen[u]) continue;
            seen[u] = 1;
            ++checks;
            beam_offer(beam, &bn, L, head_dist(q, heads + (int64_t)u * d, d, metric), u);
        }
    }
    int32_t m = nprobe < bn ? nprobe : bn;
    for (int32_t i = 0; i < m; ++i) out[i] = (int32_t)beam[i].id;
    if (checks_out) *checks_out = checks;
    free(seen);
    free(expanded);
    free(beam);
    return m;
}

/* seeds_stride 0: every query starts from the same S seeds; otherwise query
 * i starts from seeds[i * seeds_stride, + S) (its own entry vertices). */
void or_graph_probe(const float *queries, int64_t nq, int32_t d, const double *heads, int32_t nlist,
                    const int32_t *adj, int32_t R, const int32_t *seeds, int32_t S, int32_t seeds_stride,
                    int32_t L, int32_t max_check, int32_t nprobe, int32_t metric, int32_t *out,
                    int32_t *found, int32_t *checks)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < nq; ++i) {
        for (int32_t j = 0; j < nprobe; ++j) out[i * nprobe + j] = -1;
        found[i] = or_graph_walk(queries + i * d, d, heads, nlist, adj, R, seeds + i * seeds_stride, S, L,
                                 max_check, nprobe, metric, out + i * nprobe, checks ? checks + i : NULL);
    }
}

/* The head of each list for the navigation graph: the centroid itself for
 * float vectors; for integer vectors (uint8, int8) the centroid rounded to
 * the nearest integer (halves to even) and clipped to the type's range, a
 * point of the data's own grid. */
void or_graph_heads(const float *cent, int32_t nlist, int32_t d, int32_t raw_dtype, double *heads)
{
    for (int64_t i = 0; i < (int64_t)nlist * d; ++i) {
        double c = (double)cent[i];
        if (raw_dtype == OR_RAW_U8 || raw_dtype == OR_RAW_I8) {
            double lo = raw_dtype == OR_RAW_U8 ? 0.0 : -128.0, hi = raw_dtype == OR_RAW_U8 ? 255.0 : 127.0;
            c = nearbyint(c);
            c = c < lo ? lo : (c > hi ? hi : c);
        }
        heads[i] = c;
    }
}
