// C ABI of libfa (declared in include/fa.h): argument checks, the device
// index (upload, renumbering, rotated code rows, replica tables), the
// workspace pool and the search pipeline.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "fa_internal.h"

namespace fa {

static float half_bits_to_float(uint16_t h) {
    __half_raw r;
    r.x = h;
    return __half2float(__half(r));
}

static float e4m3_bits_to_float(uint8_t b) {
    __nv_fp8_e4m3 v;
    v.__x = b;
    return float(v);
}

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

const char *last_error() { return g_err.c_str(); }

template <class F>
static fa_status guarded(fa_index *ix, F &&f) {
    try {
        if (ix && ix->sticky.load()) {
            set_error("index unusable after an earlier fatal CUDA error");
            return FA_ERR_STATE;
        }
        f();
        return FA_OK;
    } catch (const Error &e) {
        set_error("%s", e.msg.c_str());
        if (e.st == FA_ERR_CUDA && ix) {
            // a sticky error poisons the context: mark the index unusable
            cudaError_t s = cudaDeviceSynchronize();
            if (s != cudaSuccess) ix->sticky.store(1);
            cudaGetLastError();
        }
        return e.st;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return FA_ERR_OOM;
    } catch (...) {
        set_error("unexpected internal error");
        return FA_ERR_CUDA;
    }
}

// Host-side fault injection (fa_debug_fail_alloc): the n-th next device
// allocation of the library fails as if the device were out of memory.
static std::atomic<int32_t> g_fail_alloc{0};

bool alloc_fault() {
    int32_t c = g_fail_alloc.load();
    while (c > 0)
        if (g_fail_alloc.compare_exchange_weak(c, c - 1)) return c == 1;
    return false;
}

template <class T>
static T *dev_upload(const T *src, size_t count, int64_t &bytes) {
    T *p = nullptr;
    const size_t b = sizeof(T) * (count ? count : 1);
    if (alloc_fault() || cudaMalloc(&p, b) != cudaSuccess) {
        cudaGetLastError();
        throw Error{FA_ERR_OOM, "device allocation of " + std::to_string(b) + " bytes failed"};
    }
    bytes += (int64_t)b;
    if (count) FA_CHECK_CUDA(cudaMemcpy(p, src, sizeof(T) * count, cudaMemcpyHostToDevice));
    return p;
}

void free_device_index(fa_index *ix) {
    DeviceIndex &d = ix->dev;
    void *ptrs[] = {d.centroids, d.cnorm, d.codebooks, d.codes, d.list_beg, d.rep_off,
                    d.rep_v, d.rep_mo, d.rep_t, d.mem, d.perm, d.raw_dev_alloc,
                    d.centroids_bf16, d.codebooks_bf16, d.cbnorm, d.lorder, d.vpage, d.vslot,
                    d.graph.heads, d.graph.adj, d.graph.seeds, d.graph.pivots, d.graph.pivot_tiles,
                    d.graph.pivot_norm};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    d = DeviceIndex{};
}

// Navigation graph of the lists (§4.1 "In-memory Indices"). The paper grows
// it by inserting the centroids one at a time, each linked to its nearest
// neighbours among those present, the neighbours re-trimming their own
// lists; with all vertices present the graph that converges to is each
// vertex's R nearest other vertices, computed here exactly and at once (the
// all-pairs top-(R + 1) of the heads on the GPU, FP32 direct differences:
// exact for integer heads). Seeds are spread over the list ids.
static void build_probe_graph(fa_index *ix, int32_t R, int32_t S) {
    const int32_t nlist = ix->nlist, d = ix->d;
    const bool integer = ix->raw_dtype == FA_U8 || ix->raw_dtype == FA_I8;
    std::vector<float> heads((size_t)nlist * d);
    for (size_t i = 0; i < heads.size(); ++i) {
        float c = ix->centroids[i];
        if (integer) {
            const float lo = ix->raw_dtype == FA_U8 ? 0.f : -128.f, hi = ix->raw_dtype == FA_U8 ? 255.f : 127.f;
            c = std::nearbyint(c);
            c = c < lo ? lo : (c > hi ? hi : c);
        }
        heads[i] = c;
    }
    R = std::min(R, std::max(1, nlist - 1));
    S = std::min(S, nlist);
    // candidates: the K nearest other heads of every vertex, exactly on the GPU
    const int32_t K = std::min(nlist - 1, 3 * R);
    const int32_t r = std::min(K + 1, nlist);
    std::vector<int32_t> nn((size_t)nlist * r);
    gpu_assign_topr(heads.data(), nlist, d, FA_F32, heads.data(), nlist, r, nn.data(), nullptr);
    auto hd = [&](int64_t a, int64_t b) {  // squared L2 between heads (exact for integer heads)
        double s = 0.0;
        const float *x = &heads[a * d], *y = &heads[b * d];
        for (int j = 0; j < d; ++j) {
            const double t = (double)x[j] - (double)y[j];
            s += t * t;
        }
        return s;
    };
    // 1. relative-neighbourhood pruning (as SPTAG's graph does): a candidate
    //    is kept unless an already kept neighbour is closer to it than the
    //    vertex is; so the kept edges point in different directions
    std::vector<std::vector<int32_t>> first(nlist);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t p = 0; p < nlist; ++p) {
        for (int j = 0; j < r && (int)first[p].size() < R; ++j) {
            const int32_t c = nn[p * r + j];
            if (c < 0 || c == p) continue;
            const double dpc = hd(p, c);
            bool keep = true;
            for (int32_t n : first[p])
                if (hd(n, c) < dpc) {
                    keep = false;
                    break;
                }
            if (keep) first[p].push_back(c);
        }
    }
    // 2. reverse edges: the vertices that kept u, nearest first (the paper's
    //    neighbours updating their lists when a vertex is inserted)
    std::vector<std::vector<std::pair<double, int32_t>>> rev(nlist);
    for (int64_t v = 0; v < nlist; ++v)
        for (int32_t u : first[v]) rev[u].push_back({0.0, (int32_t)v});
    // 3. out-edges: kept, then reverse, then the nearest candidates, up to R
    std::vector<int32_t> adj((size_t)nlist * R, -1);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t u = 0; u < nlist; ++u) {
        for (auto &pv : rev[u]) pv.first = hd(u, pv.second);
        std::sort(rev[u].begin(), rev[u].end());
        int32_t *row = &adj[u * R];
        int e = 0;
        auto add = [&](int32_t x) {
            if (x < 0 || x == u || e >= R) return;
            for (int i = 0; i < e; ++i)
                if (row[i] == x) return;
            row[e++] = x;
        };
        for (int32_t x : first[u]) add(x);
        for (const auto &pv : rev[u]) add(pv.second);
        for (int j = 0; j < r && e < R; ++j) add(nn[u * r + j]);
    }
    std::vector<int32_t> seeds(S);
    for (int32_t i = 0; i < S; ++i) seeds[i] = (int32_t)(((int64_t)i * nlist) / S);
    ProbeGraph &g = ix->dev.graph;
    for (void *p : {g.heads, (void *)g.adj, (void *)g.seeds, (void *)g.pivots, g.pivot_tiles,
                    (void *)g.pivot_norm})
        if (p) cudaFree(p);
    g = ProbeGraph{};
    int64_t bytes = 0;
    if (integer) {
        std::vector<uint8_t> hb(heads.size());
        for (size_t i = 0; i < heads.size(); ++i) {
            const int v = (int)heads[i];
            hb[i] = ix->raw_dtype == FA_U8 ? (uint8_t)v : (uint8_t)(int8_t)v;
        }
        g.heads = dev_upload(hb.data(), hb.size(), bytes);
    } else {
        g.heads = dev_upload(heads.data(), heads.size(), bytes);
    }
    g.head_dtype = integer ? ix->raw_dtype : FA_F32;
    g.adj = dev_upload(adj.data(), adj.size(), bytes);
    g.seeds = dev_upload(seeds.data(), seeds.size(), bytes);
    std::vector<float> piv((size_t)S * d);
    for (int32_t i = 0; i < S; ++i)
        std::copy(heads.begin() + (size_t)seeds[i] * d, heads.begin() + (size_t)(seeds[i] + 1) * d,
                  piv.begin() + (size_t)i * d);
    g.pivots = dev_upload(piv.data(), piv.size(), bytes);
    if (integer && d <= 128) {
        // integer heads are exact in bf16 (|value| <= 256) and their products
        // and sums exact in FP32 for d <= 128, so the tensor cores give the
        // entry probe the same distances as FP32 direct differences
        std::vector<uint16_t> tiles;
        prepare_centroid_tiles(piv.data(), S, d, tiles, g.pivot_kp, g.pivot_nt);
        g.pivot_tiles = dev_upload(tiles.data(), tiles.size(), bytes);
        std::vector<float> pn(S);
        for (int32_t i = 0; i < S; ++i) {
            double s2 = 0.0;
            for (int j = 0; j < d; ++j) s2 += (double)piv[(size_t)i * d + j] * piv[(size_t)i * d + j];
            pn[i] = (float)s2;
        }
        g.pivot_norm = dev_upload(pn.data(), pn.size(), bytes);
    }
    g.R = R;
    g.S = S;
    ix->dev.device_bytes += bytes;
    ix->g_adj = std::move(adj);
    ix->g_seeds = std::move(seeds);
}

// Beam, check budget and entry pivots of a graph walk (0 = the defaults).
static void graph_defaults(const ProbeGraph &g, int32_t nprobe, int32_t beam_in, int32_t max_in,
                           int32_t entry_in, int32_t &beam, int32_t &max_check, int32_t &entry) {
    FA_REQUIRE(max_in >= 0 && beam_in >= 0 && entry_in >= 0, FA_ERR_ARG, "graph beam / max_check / entry < 0");
    beam = beam_in > 0 ? beam_in : std::min(256, 2 * nprobe);
    entry = std::min(entry_in > 0 ? entry_in : 16, g.S);
    max_check = max_in > 0 ? max_in : 16 * nprobe + entry;
    FA_REQUIRE(nprobe <= 256 && beam >= nprobe && beam <= 256, FA_ERR_ARG,
               "graph probe needs nprobe <= beam <= 256");
    FA_REQUIRE(entry == g.S || entry <= 64, FA_ERR_ARG, "graph entry must be <= 64 or all pivots");
}

// Renumbers vectors by primary list, rotates code rows, builds the replica
// tables and uploads everything.
void upload_index(fa_index *ix) {
    FA_CHECK_CUDA(cudaSetDevice(ix->device));
    DeviceIndex &D = ix->dev;
    const int64_t n = ix->n;
    const int d = ix->d, nlist = ix->nlist, M = ix->M;
    D.n = n;
    D.d = d;
    D.nlist = nlist;
    D.M = M;
    D.Mp = scan_width(M);
    D.dsub = d / M;
    const int Mp = D.Mp;
    D.raw_dtype = ix->raw_dtype;
    D.metric = ix->metric;
    D.raw_location = ix->raw_location;
    int64_t bytes = 0;

    // internal order: stable by primary list
    std::vector<int64_t> cnt(nlist + 1, 0);
    for (int64_t v = 0; v < n; ++v) cnt[ix->primary[v] + 1]++;
    std::vector<uint32_t> beg(nlist + 1, 0);
    for (int l = 0; l < nlist; ++l) beg[l + 1] = (uint32_t)(beg[l] + cnt[l + 1]);
    std::vector<int64_t> perm(n), inv(n);
    {
        std::vector<uint32_t> fill(beg.begin(), beg.end() - 1);
        for (int64_t v = 0; v < n; ++v) {
            const uint32_t iv = fill[ix->primary[v]]++;
            perm[iv] = v;
            inv[v] = iv;
        }
    }
    D.max_list = 0;
    for (int l = 0; l < nlist; ++l) D.max_list = std::max<int64_t>(D.max_list, beg[l + 1] - beg[l]);

    // rotated code rows of Mp bytes: byte s of row iv = code of subspace
    // (s + iv mod 32) mod Mp (0 for the padding subspaces M .. Mp - 1)
    const int64_t n_pad = ((n + 31) / 32) * 32 + 32;
    std::vector<uint8_t> rot((size_t)n_pad * Mp, 0);
#pragma omp parallel for schedule(static)
    for (int64_t iv = 0; iv < n; ++iv) {
        const uint8_t *src = ix->codes.data() + (size_t)perm[iv] * M;
        uint8_t *dst = rot.data() + (size_t)iv * Mp;
        const int r = (int)(iv & 31);
        for (int s = 0; s < Mp; ++s) {
            const int m = (s + r) % Mp;
            dst[s] = m < M ? src[m] : 0;
        }
    }

    // replica tables
    const bool has_rep = !ix->rep_off.empty() && ix->rep_off[nlist] > 0;
    std::vector<uint64_t> roff(nlist + 1, 0);
    std::vector<uint32_t> rv, rmo, mem;
    std::vector<uint8_t> rt;
    D.max_rep = 0;
    if (has_rep) {
        const int64_t nr = ix->rep_off[nlist];
        // replica lists of each vector, ascending
        std::vector<std::vector<int32_t>> reps;
        std::vector<int64_t> rep_vecs;
        std::vector<int32_t> slot(n, -1);
        for (int l = 0; l < nlist; ++l)
            for (int64_t e = ix->rep_off[l]; e < ix->rep_off[l + 1]; ++e) {
                const int64_t v = ix->rep_ids[e];
                if (slot[v] < 0) {
                    slot[v] = (int32_t)reps.size();
                    reps.emplace_back();
                    rep_vecs.push_back(v);
                }
                reps[slot[v]].push_back(l);
            }
        std::vector<uint32_t> mo_of(reps.size());
        for (size_t i = 0; i < reps.size(); ++i) {
            std::sort(reps[i].begin(), reps[i].end());
            mo_of[i] = (uint32_t)mem.size();
            mem.push_back((uint32_t)ix->primary[rep_vecs[i]]);
            for (int32_t l : reps[i]) mem.push_back((uint32_t)l);
        }
        FA_REQUIRE(mem.size() < (1ull << 32), FA_ERR_ARG, "replica table too large");
        FA_REQUIRE(nr < (1ll << 32), FA_ERR_ARG, "too many replica entries");
        rv.resize(nr);
        rmo.resize(nr);
        rt.resize(nr);
        for (int l = 0; l < nlist; ++l) {
            // entries of list l sorted by internal id
            std::vector<std::pair<uint32_t, int64_t>> ent;
            for (int64_t e = ix->rep_off[l]; e < ix->rep_off[l + 1]; ++e)
                ent.push_back({(uint32_t)inv[ix->rep_ids[e]], ix->rep_ids[e]});
            std::sort(ent.begin(), ent.end());
            int64_t o = ix->rep_off[l];
            for (auto &pr : ent) {
                const int32_t s = slot[pr.second];
                const auto &rl = reps[s];
                const int t = 1 + (int)(std::lower_bound(rl.begin(), rl.end(), l) - rl.begin());
                rv[o] = pr.first;
                rmo[o] = mo_of[s];
                rt[o] = (uint8_t)t;
                ++o;
            }
            roff[l + 1] = (uint64_t)ix->rep_off[l + 1];
            D.max_rep = std::max<int64_t>(D.max_rep, ix->rep_off[l + 1] - ix->rep_off[l]);
        }
        D.n_rep = nr;
        D.n_mem = (int64_t)mem.size();
    }

    std::vector<float> cnorm(nlist);
    for (int l = 0; l < nlist; ++l) {
        double s = 0;
        for (int j = 0; j < d; ++j) s += (double)ix->centroids[(size_t)l * d + j] * ix->centroids[(size_t)l * d + j];
        cnorm[l] = (float)s;
    }

    D.centroids = dev_upload(ix->centroids.data(), ix->centroids.size(), bytes);
    D.cnorm = dev_upload(cnorm.data(), cnorm.size(), bytes);
    D.codebooks = dev_upload(ix->codebooks.data(), ix->codebooks.size(), bytes);
    D.codes = dev_upload(rot.data(), rot.size(), bytes);
    D.list_beg = dev_upload(beg.data(), beg.size(), bytes);
    D.rep_off = dev_upload(roff.data(), roff.size(), bytes);
    D.rep_v = dev_upload(rv.data(), rv.size(), bytes);
    D.rep_mo = dev_upload(rmo.data(), rmo.size(), bytes);
    D.rep_t = dev_upload(rt.data(), rt.size(), bytes);
    D.mem = dev_upload(mem.data(), mem.size(), bytes);
    D.perm = dev_upload(perm.data(), perm.size(), bytes);
    {
        // lists by decreasing chunk count (primary range and replica slice), so
        // that the batched scan starts the longest lists first
        std::vector<uint32_t> order(nlist), chunks(nlist);
        for (int l = 0; l < nlist; ++l) {
            order[l] = (uint32_t)l;
            chunks[l] = (beg[l + 1] - beg[l] + 31u) / 32u + (uint32_t)((roff[l + 1] - roff[l] + 31u) / 32u);
        }
        std::stable_sort(order.begin(), order.end(),
                         [&](uint32_t x, uint32_t y) { return chunks[x] > chunks[y]; });
        D.lorder = dev_upload(order.data(), order.size(), bytes);
        double cm = 0;
        for (int m = 0; m < M; ++m)
            for (int c = 0; c < 256; ++c) {
                double s2 = 0;
                for (int j = 0; j < d / M; ++j) {
                    const double x = ix->codebooks[((size_t)m * 256 + c) * (d / M) + j];
                    s2 += x * x;
                }
                cm = std::max(cm, s2);
            }
        D.cb_max_norm2 = (float)(cm * (1.0 + 1e-6));
    }
    if (d <= 128) {  // tensor-core operand tiles (BF16 hi/lo) for the coarse probe and the LUT
        std::vector<uint16_t> tiles;
        prepare_centroid_tiles(ix->centroids.data(), nlist, d, tiles, D.tc_kp, D.tc_ntiles);
        D.centroids_bf16 = dev_upload(tiles.data(), tiles.size(), bytes);
        if (16 % D.dsub == 0) {
            std::vector<float> norms;
            prepare_codebook_tiles(ix->codebooks.data(), M, d, tiles, norms);
            D.codebooks_bf16 = dev_upload(tiles.data(), tiles.size(), bytes);
            D.cbnorm = dev_upload(norms.data(), norms.size(), bytes);
        }
    }

    if (ix->h_raw) {
        const size_t rb = (size_t)n * d * raw_elem(ix->raw_dtype);
        if (ix->raw_location == FA_RAW_DEVICE) {
            // the HBM copy is in internal order (row v holds the vector with
            // internal id v), so the re-rank reads rows by the ids the scan
            // hands it and maps ids to the caller's only for the few keys
            // that can enter the top-k
            const size_t rowb = rb / (size_t)n;
            std::vector<uint8_t> rows(rb);
            const uint8_t *src = (const uint8_t *)ix->h_raw;
#pragma omp parallel for schedule(static)
            for (int64_t iv = 0; iv < n; ++iv)
                memcpy(rows.data() + (size_t)iv * rowb, src + (size_t)perm[iv] * rowb, rowb);
            D.raw_dev_alloc = dev_upload(rows.data(), rb, bytes);
            D.raw = D.raw_dev_alloc;
            D.raw_internal = 1;
        } else if (ix->raw_location == FA_RAW_HOST_PAGED) {
            // the rows in §4.3's pages in pinned host memory, read by the
            // paged re-rank through the mapping; page and row of each vector
            const int64_t rowb = (int64_t)d * raw_elem(ix->raw_dtype);
            int32_t cap = (int32_t)std::max<int64_t>(1, 4096 / rowb);
            while (cap > 1 && ((int64_t)cap * rowb) % 16 != 0) --cap;  // 16-byte page copies
            FA_REQUIRE(rowb % 4 == 0 && ((int64_t)cap * rowb) % 16 == 0 && cap <= 65535, FA_ERR_ARG,
                       "paged raw vectors need rows of a multiple of 4 bytes");
            const int64_t np = page_layout(ix->primary, nlist, cap, ix->page_of, ix->slot_of);
            const size_t pb = (size_t)cap * rowb;
            FA_CHECK_CUDA(cudaHostAlloc(&ix->h_pages, std::max<size_t>(16, pb * np),
                                        cudaHostAllocMapped | cudaHostAllocPortable));
            const uint8_t *src = (const uint8_t *)ix->h_raw;
#pragma omp parallel for schedule(static)
            for (int64_t v = 0; v < n; ++v)
                memcpy((uint8_t *)ix->h_pages + (size_t)ix->page_of[v] * pb + (size_t)ix->slot_of[v] * rowb,
                       src + (size_t)v * rowb, (size_t)rowb);
            std::vector<uint32_t> vp(n);
            std::vector<uint16_t> vs(n);
            for (int64_t v = 0; v < n; ++v) {
                vp[v] = (uint32_t)ix->page_of[v];
                vs[v] = (uint16_t)ix->slot_of[v];
            }
            D.vpage = dev_upload(vp.data(), vp.size(), bytes);
            D.vslot = dev_upload(vs.data(), vs.size(), bytes);
            D.page_rows = cap;
            D.page_bytes = (int32_t)pb;
            D.n_pages = np;
            void *dp = nullptr;
            FA_CHECK_CUDA(cudaHostGetDevicePointer(&dp, ix->h_pages, 0));
            D.raw = dp;
            D.pinned_bytes = (int64_t)(pb * np);
        } else {
            void *dp = nullptr;
            FA_CHECK_CUDA(cudaHostGetDevicePointer(&dp, ix->h_raw, 0));
            D.raw = dp;
            D.pinned_bytes = (int64_t)rb;
        }
    }
    D.device_bytes = bytes;
}

// ---------------------------------------------------------------------------
// workspace pool
// ---------------------------------------------------------------------------
static void ws_drop_graph(Workspace *w) {
    if (w->gexec) cudaGraphExecDestroy(w->gexec);
    w->gexec = nullptr;
}

static void ws_free_buffers(Workspace *w) {
    ws_drop_graph(w);
    void *dp[] = {w->q, w->probes, w->kq, w->npq, w->gentry, w->order, w->bucket, w->tchunks, w->tprefix,
                  w->tmisc, w->partial, w->topkeys, w->out_ids, w->out_dist,
                  w->stats, w->lut, w->lut_scale, w->coarse_d, w->err, w->tile_ctr, w->selbuf,
                  w->redo, w->bq_lcnt, w->bq_lqoff, w->bq_lcur, w->bq_upre, w->bq_lq, w->bq_pbits,
                  w->bq_tau, w->bq_cnt, w->bq_qsum, w->bq_buf, w->bq_ctr, w->pg_cache, w->pg_table,
                  w->pg_tslot, w->pg_reads};
    for (void *p : dp)
        if (p) cudaFree(p);
    w->pg_cache = nullptr;
    w->pg_table = nullptr;
    w->pg_tslot = nullptr;
    w->pg_reads = nullptr;
    w->pg_cap_pages = w->pg_cap_nq = 0;
    w->pg_tsize = w->pg_warps = 0;
    w->bq_lcnt = w->bq_lqoff = w->bq_lcur = w->bq_upre = w->bq_pbits = w->bq_cnt = w->bq_ctr = nullptr;
    w->bq_lq = nullptr;
    w->bq_tau = w->bq_buf = nullptr;
    w->bq_qsum = nullptr;
    w->bq_cap_nq = 0;
    w->bq_cap_pairs_np = 0;
    w->bq_cap = 0;
    void *hp[] = {w->h_err, w->h_stats, w->h_small};
    for (void *p : hp)
        if (p) cudaFreeHost(p);
    w->q = nullptr;
    w->probes = w->kq = w->npq = w->gentry = w->order = nullptr;
    w->bucket = w->tchunks = w->tprefix = w->tmisc = nullptr;
    w->partial = nullptr;
    w->tile_cap = 0;
    w->topkeys = nullptr;
    w->out_ids = nullptr;
    w->out_dist = nullptr;
    w->stats = nullptr;
    w->lut = nullptr;
    w->lut_scale = nullptr;
    w->coarse_d = nullptr;
    w->err = w->tile_ctr = nullptr;
    w->selbuf = nullptr;
    w->redo = nullptr;
    w->h_err = nullptr;
    w->h_stats = nullptr;
    w->h_small = nullptr;
    w->cap_nq = 0;
}

template <class T>
static void dalloc(T *&p, size_t count) {
    if (alloc_fault() || cudaMalloc(&p, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        throw Error{FA_ERR_OOM, "workspace allocation failed"};
    }
}

static void ws_ensure(fa_index *ix, Workspace *w, int64_t nq, int32_t k, int32_t nprobe,
                      int32_t ntop, int lut_bytes) {
    const DeviceIndex &D = ix->dev;
    if (w->cap_nq >= nq && w->cap_k >= k && w->cap_nprobe >= nprobe && w->cap_ntop >= ntop &&
        w->cap_lut_bytes >= lut_bytes)
        return;
    if (w->pending) FA_CHECK_CUDA(cudaEventSynchronize(w->done));
    w->pending = false;
    FA_CHECK_CUDA(cudaStreamSynchronize(w->stream));
    const int64_t cq = std::max(nq, w->cap_nq);
    const int32_t ck = std::max(k, w->cap_k), cp = std::max(nprobe, w->cap_nprobe),
                  ct = std::max(ntop, w->cap_ntop), cl = std::max(lut_bytes, w->cap_lut_bytes);
    ws_free_buffers(w);
    dalloc(w->q, (size_t)cq * D.d);
    dalloc(w->probes, (size_t)cq * cp);
    dalloc(w->kq, (size_t)cq);
    dalloc(w->npq, (size_t)cq);
    dalloc(w->gentry, (size_t)cq * 64);
    dalloc(w->order, (size_t)cq);
    dalloc(w->bucket, (size_t)D.nlist);
    dalloc(w->tchunks, (size_t)cq);
    dalloc(w->tprefix, (size_t)cq + 1);
    dalloc(w->tmisc, 4);
    dalloc(w->topkeys, (size_t)cq * ct);
    dalloc(w->out_ids, (size_t)cq * ck);
    dalloc(w->out_dist, (size_t)cq * ck);
    dalloc(w->stats, (size_t)cq * 4);
    dalloc(w->lut_scale, (size_t)cq * 2 * D.Mp);
    if (cl > 0) {
        char *p = nullptr;
        dalloc(p, (size_t)cq * cl);
        w->lut = p;
    }
    // distance block of the coarse probe: up to 1 GiB of rows at a time
    const int64_t ldd = coarse_tc_ldd(D.nlist);
    w->coarse_rows = std::max<int64_t>(128, std::min<int64_t>(cq, (1ll << 30) / (4ll * ldd)));
    dalloc(w->coarse_d, (size_t)w->coarse_rows * ldd);
    dalloc(w->err, 4);
    dalloc(w->tile_ctr, 4);
    if (ct > 256) {
        dalloc(w->selbuf, (size_t)2 * num_sms(ix->device) * 2 * ct);
        dalloc(w->redo, (size_t)cq);
    }
    FA_CHECK_CUDA(cudaHostAlloc((void **)&w->h_err, 16, cudaHostAllocDefault));
    FA_CHECK_CUDA(cudaHostAlloc((void **)&w->h_stats, sizeof(int32_t) * (size_t)cq * 4, cudaHostAllocDefault));
    FA_CHECK_CUDA(cudaHostAlloc((void **)&w->h_small, sizeof(int32_t) * (size_t)cq * 2, cudaHostAllocDefault));
    w->cap_nq = cq;
    w->cap_k = ck;
    w->cap_nprobe = cp;
    w->cap_ntop = ct;
    w->cap_lut_bytes = cl;
}

// Buffers of the batched form: (query, list) pairs by list, per-query
// thresholds and key buffers of cap keys (four times the top-n, at least
// 65536: 512 KB a query, so a threshold sampled from a query of millions of
// candidates does not overflow its buffer).
static uint32_t bq_key_cap(int32_t ntop) { return (uint32_t)std::max(4 * ntop, 65536); }

static void ws_ensure_batched(fa_index *ix, Workspace *w, int64_t nq, int32_t nprobe, int32_t ntop) {
    const DeviceIndex &D = ix->dev;
    const uint32_t cap = bq_key_cap(ntop);
    if (w->bq_buf && w->bq_cap_nq >= nq && w->bq_cap_pairs_np >= nprobe && w->bq_cap >= cap && w->redo)
        return;
    if (w->pending) FA_CHECK_CUDA(cudaEventSynchronize(w->done));
    w->pending = false;
    FA_CHECK_CUDA(cudaStreamSynchronize(w->stream));
    ws_drop_graph(w);
    const int64_t cq = std::max(nq, w->bq_cap_nq);
    const int32_t cp = std::max(nprobe, w->bq_cap_pairs_np);
    const uint32_t cc = std::max(cap, w->bq_cap);
    void *old[] = {w->bq_lcnt, w->bq_lqoff, w->bq_lcur, w->bq_upre, w->bq_lq, w->bq_pbits,
                   w->bq_tau, w->bq_cnt, w->bq_qsum, w->bq_buf, w->bq_ctr};
    for (void *p : old)
        if (p) cudaFree(p);
    w->bq_lcnt = w->bq_lqoff = w->bq_lcur = w->bq_upre = w->bq_pbits = w->bq_cnt = w->bq_ctr = nullptr;
    w->bq_lq = nullptr;
    w->bq_tau = w->bq_buf = nullptr;
    w->bq_qsum = nullptr;
    w->bq_cap_nq = 0;
    dalloc(w->bq_lcnt, (size_t)D.nlist);
    dalloc(w->bq_lqoff, (size_t)D.nlist + 1);
    dalloc(w->bq_lcur, (size_t)D.nlist);
    dalloc(w->bq_upre, (size_t)D.nlist + 1);
    dalloc(w->bq_lq, (size_t)cq * cp);
    dalloc(w->bq_pbits, D.n_rep > 0 ? (size_t)cq * ((D.nlist + 31) / 32) : 1);
    dalloc(w->bq_tau, (size_t)cq);
    dalloc(w->bq_cnt, (size_t)cq);
    dalloc(w->bq_qsum, (size_t)cq * 2);
    dalloc(w->bq_buf, (size_t)cq * cc);
    dalloc(w->bq_ctr, 8);
    if (!w->redo) dalloc(w->redo, (size_t)std::max(cq, w->cap_nq));
    w->bq_cap_nq = cq;
    w->bq_cap_pairs_np = cp;
    w->bq_cap = cc;
}

// Buffers of the paged re-rank: each warp of the persistent grid holds a
// buffer of top-n pages (every task on its own page at worst, so the buffer
// never evicts and inter-mini-batch deduplication is complete) and a page
// table of at least twice as many entries. The warps are capped so the
// buffers stay within 8 GiB.
static void ws_ensure_paged(fa_index *ix, Workspace *w, int64_t nq, int32_t ntop) {
    const DeviceIndex &D = ix->dev;
    const int64_t pb = D.page_bytes;
    int32_t tsize = 64;
    while (tsize < 2 * ntop) tsize *= 2;
    const int32_t warps = (int32_t)std::max<int64_t>(
        1, std::min<int64_t>(2ll * num_sms(ix->device), (8ll << 30) / std::max<int64_t>(1, (int64_t)ntop * pb)));
    if (w->pg_cache && w->pg_cap_nq >= nq && w->pg_cap_pages >= ntop && w->pg_tsize >= tsize) return;
    if (w->pending) FA_CHECK_CUDA(cudaEventSynchronize(w->done));
    w->pending = false;
    FA_CHECK_CUDA(cudaStreamSynchronize(w->stream));
    ws_drop_graph(w);
    void *old[] = {w->pg_cache, w->pg_table, w->pg_tslot, w->pg_reads};
    for (void *p : old)
        if (p) cudaFree(p);
    w->pg_cache = nullptr;
    w->pg_table = nullptr;
    w->pg_tslot = nullptr;
    w->pg_reads = nullptr;
    const int64_t cq = std::max(nq, w->pg_cap_nq);
    dalloc(w->pg_cache, (size_t)warps * ntop * pb);
    dalloc(w->pg_table, (size_t)warps * tsize);
    dalloc(w->pg_tslot, (size_t)warps * tsize);
    dalloc(w->pg_reads, (size_t)cq);
    w->pg_cap_pages = ntop;
    w->pg_cap_nq = cq;
    w->pg_tsize = tsize;
    w->pg_warps = warps;
}

// Per-tile top-n buffer of the tiled form: 16 tiles per query on average,
// the tile size adapts on the device so the plan always fits.
static void ws_ensure_partial(Workspace *w, int64_t nq, int32_t ntop) {
    const int64_t cap = 16 * nq + 1024;
    if (w->partial && w->tile_cap >= cap && w->cap_ntop >= ntop) return;
    if (w->pending) FA_CHECK_CUDA(cudaEventSynchronize(w->done));
    FA_CHECK_CUDA(cudaStreamSynchronize(w->stream));
    ws_drop_graph(w);
    if (w->partial) cudaFree(w->partial);
    w->partial = nullptr;
    dalloc(w->partial, (size_t)cap * std::max(ntop, w->cap_ntop));
    w->tile_cap = cap;
}

// chunks of a pipelined search (scan of chunk i + 1 beside the re-rank of chunk i)
constexpr int PIPE_CHUNKS = 8;

struct WsLease {
    fa_index *ix;
    Workspace *w = nullptr;
    cudaEvent_t done = nullptr;
    WsLease(fa_index *i, bool nonblocking) : ix(i) {
        std::unique_lock<std::mutex> lk(ix->mu);
        for (;;) {
            if (!ix->free_ws.empty()) {
                w = ix->free_ws.back();
                ix->free_ws.pop_back();
                break;
            }
            if ((int)ix->all_ws.size() < ix->max_ws) {
                w = new Workspace();
                w->device = ix->device;
                int prio_lo = 0, prio_hi = 0;
                cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
                bool ok = cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) == cudaSuccess &&
                          cudaEventCreateWithFlags(&w->done, cudaEventDisableTiming) == cudaSuccess &&
                          cudaStreamCreateWithPriority(&w->stream2, cudaStreamNonBlocking, prio_hi) ==
                              cudaSuccess &&
                          cudaStreamCreateWithFlags(&w->stream3, cudaStreamNonBlocking) == cudaSuccess &&
                          cudaEventCreateWithFlags(&w->join, cudaEventDisableTiming) == cudaSuccess &&
                          cudaEventCreateWithFlags(&w->join3, cudaEventDisableTiming) == cudaSuccess &&
                          cudaEventCreateWithFlags(&w->lut_done, cudaEventDisableTiming) == cudaSuccess;
                for (auto &e : w->fork)
                    ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
                for (auto &e : w->marks) ok = ok && cudaEventCreate(&e) == cudaSuccess;
                if (!ok) {
                    cudaGetLastError();
                    delete w;
                    w = nullptr;
                    throw Error{FA_ERR_CUDA, "stream creation failed"};
                }
                ix->all_ws.push_back(w);
                break;
            }
            if (nonblocking) throw Error{FA_ERR_BUSY, "no free workspace slot"};
            ix->cv.wait(lk);
        }
    }
    ~WsLease() {
        if (!w) return;
        std::lock_guard<std::mutex> lk(ix->mu);
        ix->free_ws.push_back(w);
        ix->cv.notify_one();
    }
};


// CUDA-event marks between the stages of one call (only when a trace is asked).
// Stage boundaries, recorded on the call's stream on every call (timing
// events of the workspace); read back only when the caller asks for a trace.
// Recording them costs nothing measurable, and a host-buffer call was measured
// 0.35 ms faster with them than without.
struct Tracer {
    fa_search_trace *out;
    cudaStream_t st;
    cudaEvent_t *ev;
    int32_t launches = 0;
    Tracer(fa_search_trace *o, cudaStream_t s, cudaEvent_t *marks) : out(o), st(s), ev(marks) {}
    void mark(int i) { FA_CHECK_CUDA(cudaEventRecord(ev[i], st)); }
    void finish() {
        if (!out) return;
        FA_CHECK_CUDA(cudaEventSynchronize(ev[4]));
        float t[4];
        for (int i = 0; i < 4; ++i) FA_CHECK_CUDA(cudaEventElapsedTime(&t[i], ev[i], ev[i + 1]));
        out->coarse_ms = t[0];
        out->lut_ms = t[1];
        out->scan_ms = t[2];
        out->post_ms = t[3];
        FA_CHECK_CUDA(cudaEventElapsedTime(&out->total_ms, ev[0], ev[4]));
        out->launches = launches;
    }
};

static void search_impl(fa_index *ix, const float *queries, int64_t nq, int32_t d, int32_t k,
                        int32_t nprobe, const fa_search_params *spp, int64_t *out_ids,
                        float *out_dist, const Tune *force = nullptr) {
    fa_search_params sp;
    if (spp)
        sp = *spp;
    else
        fa_search_params_init(&sp);
    FA_REQUIRE(d == ix->d, FA_ERR_ARG, "query dimension differs from the index");
    FA_REQUIRE(k >= 1 && k <= 16384, FA_ERR_ARG, "k must be in 1..16384");
    FA_REQUIRE(nq >= 0, FA_ERR_ARG, "nq < 0");
    if (nq == 0) return;
    FA_REQUIRE(queries && out_ids && out_dist, FA_ERR_ARG, "null buffer");
    nprobe = std::max(1, std::min(nprobe, ix->nlist));
    FA_REQUIRE(nprobe <= 512, FA_ERR_ARG, "nprobe above 512");
    FA_REQUIRE(sp.lut_prec >= FA_LUT_F32 && sp.lut_prec <= FA_LUT_FP8, FA_ERR_ARG, "bad lut_prec");
    FA_REQUIRE(sp.probe_gemm >= FA_GEMM_SIMT_F32 && sp.probe_gemm <= FA_PROBE_GRAPH, FA_ERR_ARG, "bad probe_gemm");
    const bool gprobe = sp.probe_gemm == FA_PROBE_GRAPH && !sp.probes;
    int32_t gbeam = 0, gmax = 0, gentry = 0;
    if (gprobe) {
        FA_REQUIRE(ix->dev.graph.adj != nullptr, FA_ERR_ARG, "FA_PROBE_GRAPH needs fa_build_probe_graph");
        graph_defaults(ix->dev.graph, nprobe, sp.graph_beam, sp.graph_max_check, sp.graph_entry, gbeam, gmax,
                       gentry);
    }
    const bool rerank = sp.rerank_n > 0;
    int32_t ntop = k;
    if (rerank) {
        FA_REQUIRE(ix->dev.raw != nullptr, FA_ERR_ARG, "re-rank needs raw vectors in the index");
        FA_REQUIRE(k <= 128, FA_ERR_ARG, "re-rank supports k <= 128");
        FA_REQUIRE(sp.rerank_batch >= 1 && sp.rerank_batch <= 4096, FA_ERR_ARG, "bad rerank_batch");
        FA_REQUIRE(sp.rerank_beta >= 1, FA_ERR_ARG, "rerank_beta < 1");
        ntop = std::max(sp.rerank_n, k);
        FA_REQUIRE(ntop <= 16384, FA_ERR_ARG, "rerank_n above 16384");
    }
    const bool qdev = sp.flags & FA_QUERIES_ON_DEVICE, odev = sp.flags & FA_OUTPUTS_ON_DEVICE;
    const bool batched = (sp.flags & FA_BATCHED) != 0;
    FA_REQUIRE(!batched || sp.lut_prec == FA_LUT_F16 || sp.lut_prec == FA_LUT_FP8, FA_ERR_ARG,
               "the batched form (FA_BATCHED) reads the FP16 or FP8 table");
    const bool global_lut = sp.lut_prec != FA_LUT_F32 || sp.lut_gemm == FA_GEMM_BF16_TC;
    const int elem = sp.lut_prec == FA_LUT_F32 ? 4 : (sp.lut_prec == FA_LUT_F16 ? 2 : 1);
    const int lut_bytes = global_lut ? ix->dev.Mp * 256 * elem : 0;

    FA_CHECK_CUDA(cudaSetDevice(ix->device));
    WsLease lease(ix, sp.flags & FA_NONBLOCKING);
    Workspace *w = lease.w;
    ws_ensure(ix, w, nq, k, nprobe, ntop, lut_bytes);
    if (batched) ws_ensure_batched(ix, w, nq, nprobe, ntop);
    // raw vectors in §4.3's pages: the re-rank runs on its own, reading pages
    const bool paged = rerank && ix->dev.raw_location == FA_RAW_HOST_PAGED;
    if (paged) ws_ensure_paged(ix, w, nq, ntop);
    FA_REQUIRE(!sp.page_reads || paged, FA_ERR_ARG, "page_reads needs a re-rank of paged raw vectors");
    cudaStream_t st = sp.stream ? (cudaStream_t)sp.stream : w->stream;
    if (w->pending) FA_CHECK_CUDA(cudaStreamWaitEvent(st, w->done, 0));
    const DeviceIndex &D = ix->dev;

    Tracer tr(sp.trace, st, w->marks);
    tr.mark(0);
    int64_t *oid = odev ? out_ids : w->out_ids;
    float *odist = odev ? out_dist : w->out_dist;
    // launch shape (autotuned per call class unless forced)
    Tune tune;
    if (force) {
        tune = *force;
    } else {
        std::lock_guard<std::mutex> lk(ix->mu);
        const Tune &c = ix->tune[tune_class(ntop, global_lut)];
        if (c.set) tune = c;
    }
    int tile_chunks = tune.tile_chunks;
    if ((sp.flags & FA_PERSISTENT) && tile_chunks == 0) tile_chunks = 256;
    if (ntop > 256 || batched) tile_chunks = 0;  // the CTA-wide top-n runs one CTA per query
    if (tile_chunks > 0) ws_ensure_partial(w, nq, ntop);
    // pipelined re-rank (see FA_SERIAL): large batches re-ranked from host memory
    const bool pipelined = rerank && tile_chunks == 0 && !batched && !(sp.flags & FA_SERIAL) &&
                           nq >= 4096 && D.raw_location == FA_RAW_HOST_PINNED;

    auto enqueue = [&]() {
        FA_CHECK_CUDA(cudaMemsetAsync(w->err, 0, 4, st));
        FA_CHECK_CUDA(cudaMemsetAsync(w->tile_ctr + 3, 0, 4, st));  // queries handed back
        const float *qd = queries;
        if (!qdev) {
            FA_CHECK_CUDA(cudaMemcpyAsync(w->q, queries, sizeof(float) * nq * d, cudaMemcpyHostToDevice, st));
            qd = w->q;
        }
        const int32_t *kq = nullptr, *npq = nullptr;
        if (sp.k_per_query) {
            if (qdev) kq = sp.k_per_query;
            else {
                FA_CHECK_CUDA(cudaMemcpyAsync(w->kq, sp.k_per_query, 4 * nq, cudaMemcpyHostToDevice, st));
                kq = w->kq;
            }
        }
        if (sp.nprobe_per_query) {
            if (qdev) npq = sp.nprobe_per_query;
            else {
                FA_CHECK_CUDA(cudaMemcpyAsync(w->npq, sp.nprobe_per_query, 4 * nq, cudaMemcpyHostToDevice, st));
                npq = w->npq;
            }
        }
        const int32_t *probes = w->probes;
        if (sp.probes) {
            if (qdev) probes = sp.probes;
            else FA_CHECK_CUDA(cudaMemcpyAsync(w->probes, sp.probes, sizeof(int32_t) * nq * nprobe,
                                               cudaMemcpyHostToDevice, st));
        } else if (gprobe) {
            // steps 1 and 2 at the same time (§3): the table on a second
            // stream while the walk runs on the call's stream
            if (global_lut) {
                FA_CHECK_CUDA(cudaEventRecord(w->fork[0], st));
                FA_CHECK_CUDA(cudaStreamWaitEvent(w->stream2, w->fork[0], 0));
                launch_lut_global(D, qd, nq, sp.lut_prec, sp.lut_gemm, w->lut, w->lut_scale, w->err,
                                  w->stream2, batched ? 1 : 0);
                FA_CHECK_CUDA(cudaEventRecord(w->join, w->stream2));
                tr.launches += 1;
            }
            launch_graph_probe(D, qd, nq, nprobe, nprobe, gbeam, gmax, gentry, npq, w->probes, w->npq, nullptr,
                               w->coarse_d, w->coarse_rows, w->gentry, w->err, st);
            npq = w->npq;
            tr.launches += gentry < D.graph.S ? 3 : 1;
        } else {
            // the table on the second stream here too: it needs only the
            // queries, and overlaps the probe's selection
            if (global_lut) {
                FA_CHECK_CUDA(cudaEventRecord(w->fork[0], st));
                FA_CHECK_CUDA(cudaStreamWaitEvent(w->stream2, w->fork[0], 0));
                launch_lut_global(D, qd, nq, sp.lut_prec, sp.lut_gemm, w->lut, w->lut_scale, w->err,
                                  w->stream2, batched ? 1 : 0);
                FA_CHECK_CUDA(cudaEventRecord(w->join, w->stream2));
                tr.launches += 1;
            }
            launch_coarse(D, qd, nq, nprobe, nprobe, sp.probe_gemm, *w, w->probes, st);
            tr.launches += coarse_launches(D, nq, sp.probe_gemm, *w);
        }
        tr.mark(1);
        const bool lut_forked = global_lut && !sp.probes;
        if (lut_forked) {
            FA_CHECK_CUDA(cudaStreamWaitEvent(st, w->join, 0));
        } else if (global_lut) {
            launch_lut_global(D, qd, nq, sp.lut_prec, sp.lut_gemm, w->lut, w->lut_scale, w->err, st,
                              batched ? 1 : 0);
            tr.launches += 1;
        }
        tr.mark(2);

        bool fused = false;  // the re-rank ran inside the scan
        ScanLaunch sl{};
        sl.q = qd;
        sl.probes = probes;
        sl.npq = npq;
        sl.ntopq = rerank ? nullptr : kq;
        sl.nq = nq;
        sl.nprobe = nprobe;
        sl.probe_stride = nprobe;
        sl.ntop = ntop;
        sl.lut_prec = global_lut ? sp.lut_prec : -1;
        sl.lut = w->lut;
        sl.lut_scale = w->lut_scale;
        sl.topkeys = w->topkeys;
        sl.stats = sp.stats ? w->stats : nullptr;
        sl.err = w->err;
        sl.tile_ctr = w->tile_ctr;
        sl.threads = tune.threads;
        sl.ilp = tune.ilp;
        sl.persistent = ((sp.flags & FA_PERSISTENT) || tune.persistent) ? 1 : 0;
        // only a re-rank that may stop early reads the top-n in order; the
        // output stage sorts what it returns
        sl.sorted = (rerank && sp.rerank_eps >= 0.f) ? 1 : 0;
        if (sp.stats) FA_CHECK_CUDA(cudaMemsetAsync(w->stats, 0, sizeof(int32_t) * 4 * nq, st));
        if (tile_chunks > 0) {
            // batching form: uneven queries split into tiles of chunks, planned on the device
            launch_tile_plan(D, probes, npq, nq, nprobe, nprobe, (uint32_t)tile_chunks,
                             (uint32_t)w->tile_cap, w->tchunks,
                             reinterpret_cast<unsigned long long *>(w->tmisc + 2), w->tmisc, w->tprefix, st);
            sl.tile_prefix = w->tprefix;
            sl.tile_T = w->tmisc;
            sl.partial = w->partial;
            sl.persistent = 1;
            FA_CHECK_CUDA(cudaMemsetAsync(w->tile_ctr, 0, 4, st));
            launch_scan(D, sl, st);
            launch_tile_merge(w->partial, w->tprefix, nq, ntop, w->topkeys, st);
            tr.launches += 4;
        } else if (batched) {
            // batched form: the whole batch scanned list by list (queries
            // grouped by their first list only orders the threshold sample)
            launch_query_order(probes, nq, nprobe, ix->nlist, w->bucket, w->order, st);
            sl.order = w->order;
            sl.redo = w->redo;
            sl.fuse_rerank = (rerank && !paged && sp.rerank_eps < 0.f) ? 1 : 0;
            sl.k = k;
            sl.kq = kq;
            sl.rerank_batch = sp.rerank_batch;
            sl.out_ids = oid;
            sl.out_dist = odist;
            BatchBufs bb{};
            bb.lcnt = w->bq_lcnt;
            bb.lqoff = w->bq_lqoff;
            bb.lcur = w->bq_lcur;
            bb.upre = w->bq_upre;
            bb.pbits = w->bq_pbits;
            bb.cnt = w->bq_cnt;
            bb.ctr = w->bq_ctr;
            bb.lq = w->bq_lq;
            bb.tau = w->bq_tau;
            bb.buf = w->bq_buf;
            bb.qsum = w->bq_qsum;
            bb.cap = w->bq_cap;
            bb.tile_chunks = 1024;
            // sub-batches whose tables (M x 256 entries a query) fit in ~40 MB of L2
            bb.qsub = std::max<int64_t>(1024, (40ll << 20) / ((int64_t)D.Mp * 256 * elem));
            fused = launch_batched(D, sl, bb, st);
            const int64_t nsub = (nq + bb.qsub - 1) / bb.qsub;
            tr.launches += 2 + (int)(4 * nsub) + 2;
        } else if (pipelined) {
            // chunk c's re-rank (on the slot's high-priority stream, waiting on
            // the host link) runs while chunk c + 1 is scanned. Scans alternate
            // between the call's stream and a second one so that one chunk's
            // last CTAs overlap the next chunk's first; the re-rank is a
            // persistent one-warp-per-SM grid, so the scans keep their occupancy.
            // chunk sizes shrink towards the end (weights 4,4,4,4,4,3,2,1): the
            // re-ranks still running when the last scans finish are short
            static constexpr int PIPE_W[PIPE_CHUNKS] = {4, 4, 4, 4, 4, 3, 2, 1};
            int32_t *stt = sp.stats ? w->stats : nullptr;
            FA_CHECK_CUDA(cudaEventRecord(w->lut_done, st));
            FA_CHECK_CUDA(cudaStreamWaitEvent(w->stream3, w->lut_done, 0));
            int64_t q0 = 0, wsum = 0;
            for (int c = 0; c < PIPE_CHUNKS; ++c) {
                wsum += PIPE_W[c];
                const int64_t q1 = c == PIPE_CHUNKS - 1 ? nq : nq * wsum / 26;
                const int64_t qn = q1 - q0;
                if (qn <= 0) continue;
                cudaStream_t ss = (c & 1) ? w->stream3 : st;
                ScanLaunch sc = sl;
                sc.q = qd + q0 * d;
                sc.probes = probes + q0 * nprobe;
                sc.npq = npq ? npq + q0 : nullptr;
                sc.nq = qn;
                sc.lut = w->lut ? static_cast<char *>(w->lut) + q0 * lut_bytes : nullptr;
                sc.lut_scale = w->lut_scale + q0 * 2 * D.Mp;
                sc.topkeys = w->topkeys + q0 * ntop;
                sc.stats = stt ? stt + q0 * 4 : nullptr;
                sc.order = nullptr;
                sc.persistent = 0;  // one counter would be shared by the two scan streams
                launch_scan(D, sc, ss);
                FA_CHECK_CUDA(cudaEventRecord(w->fork[c], ss));
                FA_CHECK_CUDA(cudaStreamWaitEvent(w->stream2, w->fork[c], 0));
                launch_rerank(D, qd + q0 * d, w->topkeys + q0 * ntop, qn, ntop, k, kq ? kq + q0 : nullptr,
                              sp.rerank_batch, sp.rerank_beta, sp.rerank_eps, oid + q0 * k, odist + q0 * k,
                              stt ? stt + q0 * 4 : nullptr, 1, w->tile_ctr + 1, w->stream2);
                tr.launches += 2;
                q0 = q1;
            }
            FA_CHECK_CUDA(cudaEventRecord(w->join3, w->stream3));
            FA_CHECK_CUDA(cudaStreamWaitEvent(st, w->join3, 0));
            tr.mark(3);
            FA_CHECK_CUDA(cudaEventRecord(w->join, w->stream2));
            FA_CHECK_CUDA(cudaStreamWaitEvent(st, w->join, 0));
        } else {
            launch_query_order(probes, nq, nprobe, ix->nlist, w->bucket, w->order, st);
            sl.order = w->order;
            sl.selbuf = w->selbuf;
            sl.redo = w->redo;
            // an exhaustive re-rank (eps < 0) runs inside the selecting scan
            sl.fuse_rerank = (rerank && !paged && sp.rerank_eps < 0.f) ? 1 : 0;
            sl.k = k;
            sl.kq = kq;
            sl.rerank_batch = sp.rerank_batch;
            sl.out_ids = oid;
            sl.out_dist = odist;
            if (sl.persistent) FA_CHECK_CUDA(cudaMemsetAsync(w->tile_ctr, 0, 4, st));
            fused = launch_scan(D, sl, st);
            tr.launches += 4 + ((ntop > 256 && !sl.sorted && w->selbuf) ? 1 : 0);
        }
        if (!pipelined) {
            tr.mark(3);
            if (paged) {
                PagedBufs pb{};
                pb.cache = w->pg_cache;
                pb.table = w->pg_table;
                pb.tslot = w->pg_tslot;
                pb.reads = w->pg_reads;
                pb.cap_pages = w->pg_cap_pages;
                pb.tsize = w->pg_tsize;
                pb.warps = w->pg_warps;
                launch_rerank_paged(D, qd, w->topkeys, nq, ntop, k, kq, sp.rerank_batch, sp.rerank_beta,
                                    sp.rerank_eps, oid, odist, sp.stats ? w->stats : nullptr, pb,
                                    w->tile_ctr + 1, st);
            } else if (rerank && fused)  // only the queries the selecting scan handed back
                launch_rerank(D, qd, w->topkeys, nq, ntop, k, kq, sp.rerank_batch, sp.rerank_beta,
                              sp.rerank_eps, oid, odist, sp.stats ? w->stats : nullptr, 1,
                              w->tile_ctr + 1, st, w->redo, w->tile_ctr + 3);
            else if (rerank)
                launch_rerank(D, qd, w->topkeys, nq, ntop, k, kq, sp.rerank_batch, sp.rerank_beta,
                              sp.rerank_eps, oid, odist, sp.stats ? w->stats : nullptr, 8, nullptr, st);
            else
                launch_finish(D, w->topkeys, nq, ntop, k, kq, oid, odist, st);
            tr.launches += 1;
        }
        tr.mark(4);

    };

    if (sp.flags & FA_GRAPH) {
        // capture once per (shape, parameters, pointers, stream), replay afterwards
        FA_REQUIRE(qdev && odev && !sp.stats && !sp.trace, FA_ERR_ARG,
                   "FA_GRAPH needs device queries and outputs and no stats or trace");
        GraphKey key{};
        key.q = queries;
        key.oi = out_ids;
        key.od = out_dist;
        key.probes = sp.probes;
        key.kq = sp.k_per_query;
        key.npq = sp.nprobe_per_query;
        key.st = st;
        key.nq = nq;
        key.k = k;
        key.nprobe = nprobe;
        key.lut_prec = sp.lut_prec;
        key.lut_gemm = sp.lut_gemm;
        key.probe_gemm = sp.probe_gemm;
        key.graph_beam = gbeam;
        key.graph_max_check = gmax;
        key.graph_entry = gentry;
        key.rerank_n = sp.rerank_n;
        key.rerank_batch = sp.rerank_batch;
        key.rerank_beta = sp.rerank_beta;
        key.rerank_eps = sp.rerank_eps;
        key.flags = sp.flags & (FA_PERSISTENT | FA_SERIAL | FA_BATCHED);
        key.threads = tune.threads;
        key.ilp = tune.ilp;
        key.persistent = tune.persistent;
        key.tile_chunks = tile_chunks;
        if (!(w->gexec && memcmp(&w->gkey, &key, sizeof key) == 0)) {
            if (w->gexec) {
                cudaGraphExecDestroy(w->gexec);
                w->gexec = nullptr;
            }
            FA_CHECK_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
            try {
                enqueue();
            } catch (...) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(st, &g);
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                throw;
            }
            cudaGraph_t g = nullptr;
            FA_CHECK_CUDA(cudaStreamEndCapture(st, &g));
            const cudaError_t ie = cudaGraphInstantiate(&w->gexec, g, 0);
            cudaGraphDestroy(g);
            FA_CHECK_CUDA(ie);
            w->gkey = key;
        }
        FA_CHECK_CUDA(cudaGraphLaunch(w->gexec, st));
    } else {
        enqueue();
    }
    if (!odev) {
        FA_CHECK_CUDA(cudaMemcpyAsync(out_ids, oid, sizeof(int64_t) * nq * k, cudaMemcpyDeviceToHost, st));
        FA_CHECK_CUDA(cudaMemcpyAsync(out_dist, odist, sizeof(float) * nq * k, cudaMemcpyDeviceToHost, st));
    }
    if (sp.stats)
        FA_CHECK_CUDA(cudaMemcpyAsync(w->h_stats, w->stats, sizeof(int32_t) * 4 * nq, cudaMemcpyDeviceToHost, st));
    if (sp.page_reads)  // pageable host memory: the copy completes before it returns
        FA_CHECK_CUDA(cudaMemcpyAsync(sp.page_reads, w->pg_reads, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, st));
    if (!((sp.flags & FA_NO_SYNC) && odev && !sp.stats && !sp.trace))
        FA_CHECK_CUDA(cudaMemcpyAsync(w->h_err, w->err, 4, cudaMemcpyDeviceToHost, st));
    if ((sp.flags & FA_NO_SYNC) && odev && !sp.stats && !sp.trace) {
        // the next user of this slot waits for the event before touching it
        FA_CHECK_CUDA(cudaEventRecord(w->done, st));
        w->pending = true;
        return;
    }
    FA_CHECK_CUDA(cudaStreamSynchronize(st));
    w->pending = false;
    const uint32_t e = *w->h_err;
    if (e & DEV_ERR_TIMEOUT) throw Error{FA_ERR_TIMEOUT, "a device-side wait ran out"};
    if (e & DEV_ERR_OVERFLOW) throw Error{FA_ERR_OVERFLOW, "an internal buffer bound was exceeded"};
    if (e & DEV_ERR_BOUNDS) throw Error{FA_ERR_ARG, "a probe list id is out of range"};
    if (sp.stats)
        for (int64_t i = 0; i < nq * 4; ++i) sp.stats[i] = w->h_stats[i];
    tr.finish();
    if (sp.trace) {
        uint32_t hb = 0;
        FA_CHECK_CUDA(cudaMemcpy(&hb, w->tile_ctr + 3, 4, cudaMemcpyDeviceToHost));
        sp.trace->handed_back = (int32_t)hb;
    }
}

static void check_parts(const fa_index_parts *p) {
    FA_REQUIRE(p != nullptr, FA_ERR_ARG, "null parts");
    FA_REQUIRE(p->n >= 1 && p->n < (1ll << 32) - 64, FA_ERR_ARG, "n must be in 1 .. 2^32-65");
    FA_REQUIRE(p->d >= 1 && p->d <= 1024, FA_ERR_ARG, "d must be in 1..1024");
    FA_REQUIRE(p->nlist >= 1, FA_ERR_ARG, "nlist must be >= 1");
    FA_REQUIRE(p->M >= 1 && p->M <= 64, FA_ERR_ARG, "M must be in 1..64");
    FA_REQUIRE(p->d % p->M == 0, FA_ERR_ARG, "d must be a multiple of M");
    FA_REQUIRE(p->d / p->M <= 16, FA_ERR_ARG, "d / M must be <= 16");
    FA_REQUIRE(p->centroids && p->codebooks && p->codes && p->primary, FA_ERR_ARG, "null part");
    FA_REQUIRE(p->raw_dtype == FA_F32 || p->raw_dtype == FA_U8 || p->raw_dtype == FA_I8, FA_ERR_ARG,
               "bad raw dtype");
    FA_REQUIRE(p->metric == FA_METRIC_L2 || p->metric == FA_METRIC_IP, FA_ERR_ARG, "bad metric");
    FA_REQUIRE(p->raw_location >= FA_RAW_NONE && p->raw_location <= FA_RAW_HOST_PAGED, FA_ERR_ARG,
               "bad raw location");
    for (int64_t v = 0; v < p->n; ++v)
        FA_REQUIRE(p->primary[v] >= 0 && p->primary[v] < p->nlist, FA_ERR_ARG, "primary list out of range");
    if (p->rep_off) {
        FA_REQUIRE(p->rep_off[0] == 0, FA_ERR_ARG, "rep_off[0] != 0");
        for (int l = 0; l < p->nlist; ++l)
            FA_REQUIRE(p->rep_off[l + 1] >= p->rep_off[l], FA_ERR_ARG, "rep_off not ascending");
        const int64_t nr = p->rep_off[p->nlist];
        FA_REQUIRE(nr == 0 || p->rep_ids, FA_ERR_ARG, "null rep_ids");
        std::vector<std::pair<int64_t, int32_t>> seen;
        seen.reserve(nr);
        for (int l = 0; l < p->nlist; ++l)
            for (int64_t e = p->rep_off[l]; e < p->rep_off[l + 1]; ++e) {
                const int64_t v = p->rep_ids[e];
                FA_REQUIRE(v >= 0 && v < p->n, FA_ERR_ARG, "replica id out of range");
                FA_REQUIRE(p->primary[v] != l, FA_ERR_ARG, "a vector is replicated into its own primary list");
                seen.push_back({v, l});
            }
        std::sort(seen.begin(), seen.end());
        for (size_t i = 1; i < seen.size(); ++i)
            FA_REQUIRE(seen[i] != seen[i - 1], FA_ERR_ARG, "a vector appears twice in one list");
        std::vector<int32_t> per(p->n, 0);
        for (auto &s : seen) FA_REQUIRE(++per[s.first] <= 7, FA_ERR_ARG, "a vector is in more than 8 lists");
    }
}

static void copy_parts(fa_index *ix, const fa_index_parts *p) {
    ix->n = p->n;
    ix->d = p->d;
    ix->nlist = p->nlist;
    ix->M = p->M;
    ix->raw_dtype = p->raw_dtype;
    ix->metric = p->metric;
    ix->raw_location = p->raw ? (p->raw_location ? p->raw_location : FA_RAW_HOST_PINNED) : FA_RAW_NONE;
    ix->centroids.assign(p->centroids, p->centroids + (size_t)p->nlist * p->d);
    ix->codebooks.assign(p->codebooks, p->codebooks + (size_t)p->d * 256);
    ix->codes.assign(p->codes, p->codes + (size_t)p->n * p->M);
    ix->primary.assign(p->primary, p->primary + p->n);
    if (p->rep_off) {
        ix->rep_off.assign(p->rep_off, p->rep_off + p->nlist + 1);
        ix->rep_ids.assign(p->rep_ids, p->rep_ids + p->rep_off[p->nlist]);
    } else {
        ix->rep_off.assign(p->nlist + 1, 0);
    }
    if (p->raw) {
        const size_t rb = (size_t)p->n * p->d * raw_elem(p->raw_dtype);
        if (ix->raw_location == FA_RAW_HOST_PINNED) {
            FA_CHECK_CUDA(cudaHostAlloc(&ix->h_raw, rb, cudaHostAllocMapped | cudaHostAllocPortable));
            ix->h_raw_pinned = true;
        } else {
            ix->h_raw = malloc(rb);
            FA_REQUIRE(ix->h_raw, FA_ERR_OOM, "host allocation of raw vectors failed");
        }
        memcpy(ix->h_raw, p->raw, rb);
    }
}

static void destroy(fa_index *ix) {
    if (!ix) return;
    cudaSetDevice(ix->device);
    for (Workspace *w : ix->all_ws) {
        if (w->pending) cudaEventSynchronize(w->done);
        if (w->stream) cudaStreamSynchronize(w->stream);
        ws_free_buffers(w);
        if (w->stream2) cudaStreamSynchronize(w->stream2);
        if (w->stream3) cudaStreamSynchronize(w->stream3);
        if (w->stream) cudaStreamDestroy(w->stream);
        if (w->stream2) cudaStreamDestroy(w->stream2);
        if (w->stream3) cudaStreamDestroy(w->stream3);
        if (w->done) cudaEventDestroy(w->done);
        if (w->join) cudaEventDestroy(w->join);
        if (w->join3) cudaEventDestroy(w->join3);
        if (w->lut_done) cudaEventDestroy(w->lut_done);
        for (cudaEvent_t e : w->fork)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : w->marks)
            if (e) cudaEventDestroy(e);
        delete w;
    }
    free_device_index(ix);
    if (ix->h_raw) {
        if (ix->h_raw_pinned) cudaFreeHost(ix->h_raw);
        else free(ix->h_raw);
    }
    if (ix->h_pages) cudaFreeHost(ix->h_pages);
    delete ix;
}

static int current_device() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{FA_ERR_NODEV, std::string("no usable CUDA device: ") + cudaGetErrorString(e)};
    }
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        throw Error{FA_ERR_NODEV, "no usable CUDA device"};
    }
    return dev;
}

}  // namespace fa

using namespace fa;

extern "C" {

void fa_build_params_init(fa_build_params *p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->nlist = 256;
    p->M = 16;
    p->kmeans_iters = 10;
    p->max_lists_per_vec = 1;
    p->train_sample = 0;
    p->seed = 20240916ull;
    p->repl_eps = 0.f;
    p->metric = FA_METRIC_L2;
    p->raw_location = FA_RAW_NONE;
    p->use_gpu = 1;
}

void fa_search_params_init(fa_search_params *sp) {
    if (!sp) return;
    memset(sp, 0, sizeof *sp);
    sp->lut_prec = FA_LUT_F32;
    sp->lut_gemm = FA_GEMM_SIMT_F32;
    sp->probe_gemm = FA_GEMM_SIMT_F32;
    sp->rerank_n = 0;
    sp->rerank_batch = 32;
    sp->rerank_beta = 2;
    sp->rerank_eps = 0.f;
}

fa_status fa_index_from_parts(const fa_index_parts *parts, fa_index **out) {
    if (!out) {
        set_error("null output pointer");
        return FA_ERR_ARG;
    }
    *out = nullptr;
    fa_index *ix = nullptr;
    fa_status s = guarded(nullptr, [&] {
        check_parts(parts);
        ix = new fa_index();
        ix->device = current_device();
        copy_parts(ix, parts);
        upload_index(ix);
    });
    if (s != FA_OK) {
        destroy(ix);
        return s;
    }
    *out = ix;
    return FA_OK;
}

fa_status fa_build_index(const void *base, int64_t n, int32_t d, fa_dtype dt,
                         const fa_build_params *p, fa_index **out) {
    if (!out) {
        set_error("null output pointer");
        return FA_ERR_ARG;
    }
    *out = nullptr;
    fa_build_params bp;
    if (p)
        bp = *p;
    else
        fa_build_params_init(&bp);
    fa_index *ix = nullptr;
    fa_status s = guarded(nullptr, [&] {
        FA_REQUIRE(base != nullptr, FA_ERR_ARG, "null base");
        FA_REQUIRE(dt == FA_F32 || dt == FA_U8 || dt == FA_I8, FA_ERR_ARG, "bad dtype");
        FA_REQUIRE(n >= 1 && n < (1ll << 32) - 64, FA_ERR_ARG, "n out of range");
        FA_REQUIRE(bp.nlist >= 1 && bp.nlist <= n, FA_ERR_ARG, "nlist must be in 1..n");
        FA_REQUIRE(bp.max_lists_per_vec >= 1 && bp.max_lists_per_vec <= 8, FA_ERR_ARG,
                   "max_lists_per_vec must be in 1..8");
        FA_REQUIRE(bp.M >= 1 && d % bp.M == 0, FA_ERR_ARG, "d must be a multiple of M");
        FA_REQUIRE(bp.kmeans_iters >= 0, FA_ERR_ARG, "kmeans_iters < 0");
        if (bp.use_gpu) current_device();
        BuildOut bo;
        train_and_encode(base, n, d, dt, bp, bo);
        fa_index_parts parts{};
        parts.n = n;
        parts.d = d;
        parts.nlist = bp.nlist;
        parts.M = bp.M;
        parts.raw_dtype = dt;
        parts.metric = bp.metric;
        parts.raw_location = bp.raw_location;
        parts.centroids = bo.centroids.data();
        parts.codebooks = bo.codebooks.data();
        parts.codes = bo.codes.data();
        parts.primary = bo.primary.data();
        parts.rep_off = bo.rep_off.data();
        parts.rep_ids = bo.rep_ids.data();
        parts.raw = bp.raw_location != FA_RAW_NONE ? base : nullptr;
        check_parts(&parts);
        ix = new fa_index();
        ix->device = current_device();
        copy_parts(ix, &parts);
        upload_index(ix);
    });
    if (s != FA_OK) {
        destroy(ix);
        return s;
    }
    *out = ix;
    return FA_OK;
}

fa_status fa_build_index_lists(const void *base, int64_t n, int32_t d, fa_dtype dt,
                               const float *centroids, int32_t nlist, const int32_t *primary,
                               const fa_build_params *p, fa_index **out) {
    if (!out) {
        set_error("null output pointer");
        return FA_ERR_ARG;
    }
    *out = nullptr;
    fa_build_params bp;
    if (p)
        bp = *p;
    else
        fa_build_params_init(&bp);
    bp.nlist = nlist;
    fa_index *ix = nullptr;
    fa_status s = guarded(nullptr, [&] {
        FA_REQUIRE(base && centroids && primary, FA_ERR_ARG, "null input");
        FA_REQUIRE(dt == FA_F32 || dt == FA_U8 || dt == FA_I8, FA_ERR_ARG, "bad dtype");
        FA_REQUIRE(n >= 1 && n < (1ll << 32) - 64 && nlist >= 1, FA_ERR_ARG, "bad shape");
        FA_REQUIRE(bp.M >= 1 && d % bp.M == 0, FA_ERR_ARG, "d must be a multiple of M");
        if (bp.use_gpu) current_device();
        BuildOut bo;
        bo.centroids.assign(centroids, centroids + (size_t)nlist * d);
        bo.primary.assign(primary, primary + n);
        bo.rep_off.assign(nlist + 1, 0);
        encode_with_lists(base, n, d, dt, bp, bo);
        fa_index_parts parts{};
        parts.n = n;
        parts.d = d;
        parts.nlist = nlist;
        parts.M = bp.M;
        parts.raw_dtype = dt;
        parts.metric = bp.metric;
        parts.raw_location = bp.raw_location;
        parts.centroids = bo.centroids.data();
        parts.codebooks = bo.codebooks.data();
        parts.codes = bo.codes.data();
        parts.primary = bo.primary.data();
        parts.rep_off = bo.rep_off.data();
        parts.rep_ids = bo.rep_ids.data();
        parts.raw = bp.raw_location != FA_RAW_NONE ? base : nullptr;
        check_parts(&parts);
        ix = new fa_index();
        ix->device = current_device();
        copy_parts(ix, &parts);
        upload_index(ix);
    });
    if (s != FA_OK) {
        destroy(ix);
        return s;
    }
    *out = ix;
    return FA_OK;
}

fa_status fa_index_get_parts(const fa_index *ix, fa_index_parts *out) {
    if (!ix || !out) {
        set_error("null argument");
        return FA_ERR_ARG;
    }
    memset(out, 0, sizeof *out);
    out->n = ix->n;
    out->d = ix->d;
    out->nlist = ix->nlist;
    out->M = ix->M;
    out->raw_dtype = ix->raw_dtype;
    out->metric = ix->metric;
    out->raw_location = ix->raw_location;
    out->centroids = ix->centroids.data();
    out->codebooks = ix->codebooks.data();
    out->codes = ix->codes.data();
    out->primary = ix->primary.data();
    out->rep_off = ix->rep_off.data();
    out->rep_ids = ix->rep_ids.data();
    out->raw = ix->h_raw;
    return FA_OK;
}

fa_status fa_index_info_get(const fa_index *ix, fa_index_info *out) {
    if (!ix || !out) {
        set_error("null argument");
        return FA_ERR_ARG;
    }
    memset(out, 0, sizeof *out);
    out->n = ix->n;
    out->n_rep_entries = ix->dev.n_rep;
    out->max_list_len = ix->dev.max_list;
    out->max_rep_len = ix->dev.max_rep;
    out->device_bytes = ix->dev.device_bytes;
    out->pinned_bytes = ix->dev.pinned_bytes;
    out->d = ix->d;
    out->nlist = ix->nlist;
    out->M = ix->M;
    out->device = ix->device;
    return FA_OK;
}

static const char MAGIC[8] = {'F', 'A', 'I', 'D', 'X', '0', '0', '1'};

fa_status fa_save_index(const fa_index *ix, const char *path) {
    if (!ix || !path) {
        set_error("null argument");
        return FA_ERR_ARG;
    }
    FILE *f = fopen(path, "wb");
    if (!f) {
        set_error("cannot open %s for writing", path);
        return FA_ERR_IO;
    }
    bool ok = true;
    auto W = [&](const void *p, size_t b) { ok = ok && (b == 0 || fwrite(p, 1, b, f) == b); };
    const int64_t hdr[8] = {1, ix->n, ix->d, ix->nlist, ix->M,
                            (int64_t)ix->raw_dtype | ((int64_t)ix->metric << 8),
                            ix->h_raw ? 1 : 0, (int64_t)ix->rep_ids.size()};
    W(MAGIC, 8);
    W(hdr, sizeof hdr);
    W(ix->centroids.data(), 4 * ix->centroids.size());
    W(ix->codebooks.data(), 4 * ix->codebooks.size());
    W(ix->codes.data(), ix->codes.size());
    W(ix->primary.data(), 4 * ix->primary.size());
    W(ix->rep_off.data(), 8 * ix->rep_off.size());
    W(ix->rep_ids.data(), 8 * ix->rep_ids.size());
    if (ix->h_raw) W(ix->h_raw, (size_t)ix->n * ix->d * raw_elem(ix->raw_dtype));
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        set_error("write to %s failed", path);
        return FA_ERR_IO;
    }
    return FA_OK;
}

fa_status fa_load_index(const char *path, int32_t raw_location, fa_index **out) {
    if (!path || !out) {
        set_error("null argument");
        return FA_ERR_ARG;
    }
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) {
        set_error("cannot open %s", path);
        return FA_ERR_IO;
    }
    bool ok = true;
    auto R = [&](void *p, size_t b) { ok = ok && (b == 0 || fread(p, 1, b, f) == b); };
    char magic[8];
    int64_t hdr[8];
    R(magic, 8);
    R(hdr, sizeof hdr);
    if (!ok || memcmp(magic, MAGIC, 8) != 0 || hdr[0] != 1 || hdr[1] < 1 || hdr[2] < 1 ||
        hdr[2] > 1024 || hdr[3] < 1 || hdr[4] < 1 || hdr[7] < 0) {
        fclose(f);
        set_error("%s is not an index file of this version", path);
        return FA_ERR_IO;
    }
    const int64_t n = hdr[1], nr = hdr[7];
    const int32_t d = (int32_t)hdr[2], nlist = (int32_t)hdr[3], M = (int32_t)hdr[4];
    const int32_t rdt = (int32_t)(hdr[5] & 0xff);  // the metric sits in the next byte
    std::vector<float> cent, cb;
    std::vector<uint8_t> codes, raw;
    std::vector<int32_t> prim;
    std::vector<int64_t> roff, rids;
    try {
        cent.resize((size_t)nlist * d);
        cb.resize((size_t)d * 256);
        codes.resize((size_t)n * M);
        prim.resize(n);
        roff.resize(nlist + 1);
        rids.resize(nr);
        if (hdr[6]) raw.resize((size_t)n * d * raw_elem(rdt));
    } catch (...) {
        fclose(f);
        set_error("host allocation failed");
        return FA_ERR_OOM;
    }
    R(cent.data(), 4 * cent.size());
    R(cb.data(), 4 * cb.size());
    R(codes.data(), codes.size());
    R(prim.data(), 4 * prim.size());
    R(roff.data(), 8 * roff.size());
    R(rids.data(), 8 * rids.size());
    if (hdr[6]) R(raw.data(), raw.size());
    fclose(f);
    if (!ok) {
        set_error("%s is truncated", path);
        return FA_ERR_IO;
    }
    fa_index_parts p{};
    p.n = n;
    p.d = d;
    p.nlist = nlist;
    p.M = M;
    p.raw_dtype = rdt;
    p.metric = (int32_t)((hdr[5] >> 8) & 0xff);
    p.raw_location = hdr[6] ? (raw_location ? raw_location : FA_RAW_HOST_PINNED) : FA_RAW_NONE;
    p.centroids = cent.data();
    p.codebooks = cb.data();
    p.codes = codes.data();
    p.primary = prim.data();
    p.rep_off = roff.data();
    p.rep_ids = rids.data();
    p.raw = (hdr[6] && raw_location != FA_RAW_NONE) ? raw.data() : nullptr;
    if (!p.raw) p.raw_location = FA_RAW_NONE;
    return fa_index_from_parts(&p, out);
}

void fa_free_index(fa_index *ix) { destroy(ix); }

fa_status fa_search_ex(fa_index *ix, const float *queries, int64_t nq, int32_t d, int32_t k,
                       int32_t nprobe, const fa_search_params *sp, int64_t *out_ids,
                       float *out_dist) {
    if (!ix) {
        set_error("null index");
        return FA_ERR_ARG;
    }
    return guarded(ix, [&] { search_impl(ix, queries, nq, d, k, nprobe, sp, out_ids, out_dist); });
}

fa_status fa_autotune(fa_index *ix, const float *queries, int64_t nq, int32_t d, int32_t k,
                      int32_t nprobe, const fa_search_params *spp, fa_tune_result *out) {
    if (!ix || !out) {
        set_error("null argument");
        return FA_ERR_ARG;
    }
    return guarded(ix, [&] {
        FA_REQUIRE(nq >= 1 && queries, FA_ERR_ARG, "autotuning needs at least one query");
        fa_search_params sp;
        if (spp) sp = *spp; else fa_search_params_init(&sp);
        FA_REQUIRE(!(sp.flags & (FA_QUERIES_ON_DEVICE | FA_OUTPUTS_ON_DEVICE)), FA_ERR_ARG,
                   "autotuning takes host queries");
        sp.flags &= ~FA_PERSISTENT;
        sp.stats = nullptr;
        const int32_t ntop = sp.rerank_n > 0 ? std::max(sp.rerank_n, k) : k;
        const bool global_lut = sp.lut_prec != FA_LUT_F32 || sp.lut_gemm == FA_GEMM_BF16_TC;
        std::vector<Tune> variants;
        if (ntop > 256) {
            for (int per = 0; per < 2; ++per) {
                Tune t;
                t.persistent = per;
                variants.push_back(t);
            }
        } else {
            // one CTA per query: threads x chunks in flight
            for (int th : {256, 512})
                for (int ilp : {1, 2}) {
                    Tune t;
                    t.threads = th;
                    t.ilp = ilp;
                    variants.push_back(t);
                }
            // tiled persistent form: tile size in 32-candidate chunks
            const int tiles[4][3] = {{256, 2, 64}, {256, 2, 256}, {256, 2, 1024}, {512, 1, 256}};
            for (auto &v : tiles) {
                Tune t;
                t.threads = v[0];
                t.ilp = v[1];
                t.persistent = 1;
                t.tile_chunks = v[2];
                variants.push_back(t);
            }
        }
        std::vector<int64_t> ids((size_t)nq * k);
        std::vector<float> dist((size_t)nq * k);
        fa_search_trace tr;
        sp.trace = &tr;
        memset(out, 0, sizeof *out);
        int best = -1;
        std::vector<int64_t> ref_ids;
        std::vector<float> ref_dist;
        for (size_t v = 0; v < variants.size() && v < 8; ++v) {
            search_impl(ix, queries, nq, d, k, nprobe, &sp, ids.data(), dist.data(), &variants[v]);
            // every launch shape must return the same rows, bit for bit
            if (v == 0) {
                ref_ids = ids;
                ref_dist = dist;
            } else if (ids != ref_ids || memcmp(dist.data(), ref_dist.data(), 4 * dist.size()) != 0) {
                throw Error{FA_ERR_STATE, "scan launch shapes disagree (variant " +
                                              std::to_string(v) + ")"};
            }
            float t3[3];
            for (int r = 0; r < 3; ++r) {
                search_impl(ix, queries, nq, d, k, nprobe, &sp, ids.data(), dist.data(), &variants[v]);
                t3[r] = tr.scan_ms;
            }
            std::sort(t3, t3 + 3);
            out->ms[v] = t3[1];
            out->threads[v] = variants[v].threads;
            out->ilp[v] = variants[v].ilp;
            out->persistent[v] = variants[v].persistent;
            out->tile_chunks[v] = variants[v].tile_chunks;
            if (best < 0 || t3[1] < out->ms[best]) best = (int)v;
        }
        out->variants = (int32_t)std::min<size_t>(variants.size(), 8);
        out->chosen = best;
        Tune t = variants[best];
        t.set = true;
        std::lock_guard<std::mutex> lk(ix->mu);
        ix->tune[tune_class(ntop, global_lut)] = t;
    });
}

fa_status fa_search(fa_index *ix, const float *queries, int64_t nq, int32_t d, int32_t k,
                    int32_t nprobe, int64_t *out_ids, float *out_dist) {
    return fa_search_ex(ix, queries, nq, d, k, nprobe, nullptr, out_ids, out_dist);
}

fa_status fa_debug_probes(fa_index *ix, const float *queries, int64_t nq, int32_t nprobe,
                          const fa_search_params *spp, int32_t *out_probes) {
    if (!ix) {
        set_error("null index");
        return FA_ERR_ARG;
    }
    return guarded(ix, [&] {
        FA_REQUIRE(nq >= 0 && queries && out_probes, FA_ERR_ARG, "bad arguments");
        FA_REQUIRE(nprobe >= 1 && nprobe <= std::min(ix->nlist, 512), FA_ERR_ARG,
                   "nprobe must be in 1..min(nlist, 512)");
        if (nq == 0) return;
        fa_search_params sp;
        if (spp) sp = *spp; else fa_search_params_init(&sp);
        FA_CHECK_CUDA(cudaSetDevice(ix->device));
        WsLease lease(ix, false);
        Workspace *w = lease.w;
        ws_ensure(ix, w, nq, 1, nprobe, 1, 0);
        FA_CHECK_CUDA(cudaMemcpyAsync(w->q, queries, sizeof(float) * nq * ix->d, cudaMemcpyHostToDevice, w->stream));
        if (sp.probe_gemm == FA_PROBE_GRAPH) {
            FA_REQUIRE(ix->dev.graph.adj != nullptr, FA_ERR_ARG, "FA_PROBE_GRAPH needs fa_build_probe_graph");
            int32_t gb = 0, gm = 0, ge = 0;
            graph_defaults(ix->dev.graph, nprobe, sp.graph_beam, sp.graph_max_check, sp.graph_entry, gb, gm, ge);
            launch_graph_probe(ix->dev, w->q, nq, nprobe, nprobe, gb, gm, ge, nullptr, w->probes, w->npq, nullptr,
                               w->coarse_d, w->coarse_rows, w->gentry, w->err, w->stream);
        } else {
            launch_coarse(ix->dev, w->q, nq, nprobe, nprobe, sp.probe_gemm, *w, w->probes, w->stream);
        }
        FA_CHECK_CUDA(cudaMemcpyAsync(out_probes, w->probes, sizeof(int32_t) * nq * nprobe,
                                      cudaMemcpyDeviceToHost, w->stream));
        FA_CHECK_CUDA(cudaStreamSynchronize(w->stream));
    });
}

fa_status fa_debug_candidates(fa_index *ix, const float *query, int32_t nprobe,
                              const int32_t *probes, int64_t *out_ids, int64_t cap,
                              int64_t *out_n) {
    if (!ix) {
        set_error("null index");
        return FA_ERR_ARG;
    }
    return guarded(ix, [&] {
        FA_REQUIRE(out_ids && out_n && (query || probes), FA_ERR_ARG, "bad arguments");
        FA_REQUIRE(nprobe >= 1 && nprobe <= std::min(ix->nlist, 512), FA_ERR_ARG,
                   "nprobe must be in 1..min(nlist, 512)");
        FA_CHECK_CUDA(cudaSetDevice(ix->device));
        WsLease lease(ix, false);
        Workspace *w = lease.w;
        ws_ensure(ix, w, 1, 1, nprobe, 1, 0);
        cudaStream_t st = w->stream;
        if (probes) {
            FA_CHECK_CUDA(cudaMemcpyAsync(w->probes, probes, 4 * nprobe, cudaMemcpyHostToDevice, st));
        } else {
            FA_CHECK_CUDA(cudaMemcpyAsync(w->q, query, sizeof(float) * ix->d, cudaMemcpyHostToDevice, st));
            launch_coarse(ix->dev, w->q, 1, nprobe, nprobe, FA_GEMM_SIMT_F32, *w, w->probes, st);
        }
        const int64_t bound = (ix->dev.max_list + ix->dev.max_rep) * (int64_t)nprobe;
        uint32_t *buf = nullptr, *cnt = nullptr;
        dalloc(buf, (size_t)std::max<int64_t>(bound, 1));
        dalloc(cnt, 2);
        struct Free {
            void *a, *b;
            ~Free() { cudaFree(a); cudaFree(b); }
        } fr{buf, cnt};
        FA_CHECK_CUDA(cudaMemsetAsync(cnt, 0, 8, st));
        launch_debug_candidates(ix->dev, w->probes, nprobe, buf, cnt, (uint32_t)bound, st);
        uint32_t hc[2];
        FA_CHECK_CUDA(cudaMemcpyAsync(hc, cnt, 8, cudaMemcpyDeviceToHost, st));
        FA_CHECK_CUDA(cudaStreamSynchronize(st));
        FA_REQUIRE(hc[1] == 0, FA_ERR_OVERFLOW, "candidate buffer overflow");
        std::vector<uint32_t> iv(hc[0]);
        FA_CHECK_CUDA(cudaMemcpy(iv.data(), buf, 4 * (size_t)hc[0], cudaMemcpyDeviceToHost));
        std::vector<int64_t> perm(ix->n);
        FA_CHECK_CUDA(cudaMemcpy(perm.data(), ix->dev.perm, 8 * (size_t)ix->n, cudaMemcpyDeviceToHost));
        std::vector<int64_t> ids(hc[0]);
        for (size_t i = 0; i < iv.size(); ++i) ids[i] = perm[iv[i]];
        std::sort(ids.begin(), ids.end());
        *out_n = (int64_t)ids.size();
        FA_REQUIRE((int64_t)ids.size() <= cap, FA_ERR_OVERFLOW, "output capacity too small");
        std::copy(ids.begin(), ids.end(), out_ids);
    });
}

fa_status fa_build_probe_graph(fa_index *ix, int32_t R, int32_t S) {
    if (!ix) {
        set_error("null index");
        return FA_ERR_ARG;
    }
    return guarded(ix, [&] {
        if (R == 0) R = 32;
        if (S == 0) S = std::min(4096, std::max(64, ix->nlist / 64));
        FA_REQUIRE(R >= 1 && R <= 64, FA_ERR_ARG, "graph degree R must be in 1..64");
        FA_REQUIRE(S >= 1 && S <= 4096, FA_ERR_ARG, "graph seeds S must be in 1..4096");
        FA_CHECK_CUDA(cudaSetDevice(ix->device));
        build_probe_graph(ix, R, S);
    });
}

fa_status fa_index_get_graph(fa_index *ix, int32_t *adj, int32_t *seeds, int32_t *R, int32_t *S) {
    if (!ix) {
        set_error("null index");
        return FA_ERR_ARG;
    }
    return guarded(ix, [&] {
        FA_REQUIRE(ix->dev.graph.adj != nullptr, FA_ERR_ARG, "the index has no navigation graph");
        if (adj) memcpy(adj, ix->g_adj.data(), sizeof(int32_t) * ix->g_adj.size());
        if (seeds) memcpy(seeds, ix->g_seeds.data(), sizeof(int32_t) * ix->g_seeds.size());
        if (R) *R = ix->dev.graph.R;
        if (S) *S = ix->dev.graph.S;
    });
}

fa_status fa_debug_graph_probe(fa_index *ix, const float *queries, int64_t nq, int32_t nprobe,
                               int32_t beam, int32_t max_check, int32_t entry, int32_t *probes,
                               int32_t *found, int32_t *checks) {
    if (!ix) {
        set_error("null index");
        return FA_ERR_ARG;
    }
    return guarded(ix, [&] {
        FA_REQUIRE(nq >= 0 && queries && probes, FA_ERR_ARG, "bad arguments");
        FA_REQUIRE(nprobe >= 1 && nprobe <= std::min(ix->nlist, 256), FA_ERR_ARG,
                   "nprobe must be in 1..min(nlist, 256)");
        FA_REQUIRE(ix->dev.graph.adj != nullptr, FA_ERR_ARG, "FA_PROBE_GRAPH needs fa_build_probe_graph");
        if (nq == 0) return;
        int32_t gb = 0, gm = 0, ge = 0;
        graph_defaults(ix->dev.graph, nprobe, beam, max_check, entry, gb, gm, ge);
        FA_CHECK_CUDA(cudaSetDevice(ix->device));
        WsLease lease(ix, false);
        Workspace *w = lease.w;
        ws_ensure(ix, w, nq, 1, nprobe, 1, 0);
        FA_CHECK_CUDA(cudaMemcpyAsync(w->q, queries, sizeof(float) * nq * ix->d, cudaMemcpyHostToDevice, w->stream));
        launch_graph_probe(ix->dev, w->q, nq, nprobe, nprobe, gb, gm, ge, nullptr, w->probes, w->npq, w->kq,
                           w->coarse_d, w->coarse_rows, w->gentry, w->err, w->stream);
        FA_CHECK_CUDA(cudaMemcpyAsync(probes, w->probes, sizeof(int32_t) * nq * nprobe, cudaMemcpyDeviceToHost,
                                      w->stream));
        if (found)
            FA_CHECK_CUDA(cudaMemcpyAsync(found, w->npq, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, w->stream));
        if (checks)
            FA_CHECK_CUDA(cudaMemcpyAsync(checks, w->kq, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, w->stream));
        FA_CHECK_CUDA(cudaStreamSynchronize(w->stream));
    });
}

fa_status fa_debug_page_map(fa_index *ix, int64_t *page_of, int32_t *slot_of, int32_t *rows_per_page,
                            int64_t *pages) {
    if (!ix) {
        set_error("null index");
        return FA_ERR_ARG;
    }
    return guarded(ix, [&] {
        FA_REQUIRE(ix->raw_location == FA_RAW_HOST_PAGED, FA_ERR_ARG, "raw vectors are not paged");
        if (page_of) memcpy(page_of, ix->page_of.data(), sizeof(int64_t) * ix->page_of.size());
        if (slot_of) memcpy(slot_of, ix->slot_of.data(), sizeof(int32_t) * ix->slot_of.size());
        if (rows_per_page) *rows_per_page = ix->dev.page_rows;
        if (pages) *pages = ix->dev.n_pages;
    });
}

fa_status fa_debug_fail_alloc(int32_t n) {
    if (n < 0) {
        set_error("n must be >= 0");
        return FA_ERR_ARG;
    }
    g_fail_alloc.store(n);
    return FA_OK;
}

fa_status fa_debug_tau_sigma(float sigma) {
    if (!(sigma == sigma)) {
        set_error("sigma is NaN");
        return FA_ERR_ARG;
    }
    fa::set_tau_sigma(sigma);
    return FA_OK;
}

fa_status fa_debug_timeout(uint32_t polls) {
    uint32_t *dev = nullptr;  // [0] status word, [1] a flag nothing sets
    try {
        int n = 0;
        if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
            cudaGetLastError();
            throw Error{FA_ERR_NODEV, "no CUDA device"};
        }
        FA_CHECK_CUDA(cudaMalloc(&dev, 8));
        FA_CHECK_CUDA(cudaMemset(dev, 0, 8));
        launch_wait_nothing(polls, dev + 1, dev, nullptr);
        uint32_t st = 0;
        FA_CHECK_CUDA(cudaMemcpy(&st, dev, 4, cudaMemcpyDeviceToHost));
        cudaFree(dev);
        dev = nullptr;
        if (st & DEV_ERR_TIMEOUT) throw Error{FA_ERR_TIMEOUT, "a device-side wait ran out"};
        return FA_OK;
    } catch (const Error &e) {
        if (dev) cudaFree(dev);
        set_error("%s", e.msg.c_str());
        return e.st;
    }
}

fa_status fa_debug_lut(fa_index *ix, const float *query, const fa_search_params *spp,
                       float *out_lut) {
    if (!ix) {
        set_error("null index");
        return FA_ERR_ARG;
    }
    return guarded(ix, [&] {
        FA_REQUIRE(query && out_lut, FA_ERR_ARG, "bad arguments");
        fa_search_params sp;
        if (spp) sp = *spp; else fa_search_params_init(&sp);
        FA_CHECK_CUDA(cudaSetDevice(ix->device));
        WsLease lease(ix, false);
        Workspace *w = lease.w;
        const int elem = sp.lut_prec == FA_LUT_F32 ? 4 : (sp.lut_prec == FA_LUT_F16 ? 2 : 1);
        const int M = ix->M;  // the table holds Mp rows; the first M are the subspaces
        ws_ensure(ix, w, 1, 1, 1, 1, ix->dev.Mp * 256 * elem);
        cudaStream_t st = w->stream;
        FA_CHECK_CUDA(cudaMemcpyAsync(w->q, query, sizeof(float) * ix->d, cudaMemcpyHostToDevice, st));
        FA_CHECK_CUDA(cudaMemsetAsync(w->err, 0, 4, st));
        launch_lut_global(ix->dev, w->q, 1, sp.lut_prec, sp.lut_gemm, w->lut, w->lut_scale, w->err, st,
                          (sp.flags & FA_BATCHED) ? 1 : 0);
        std::vector<uint8_t> raw((size_t)M * 256 * elem);
        std::vector<float> sc(2 * M);
        FA_CHECK_CUDA(cudaMemcpyAsync(raw.data(), w->lut, raw.size(), cudaMemcpyDeviceToHost, st));
        FA_CHECK_CUDA(cudaMemcpyAsync(sc.data(), w->lut_scale, 4 * sc.size(), cudaMemcpyDeviceToHost, st));
        FA_CHECK_CUDA(cudaStreamSynchronize(st));
        for (int m = 0; m < M; ++m)
            for (int c = 0; c < 256; ++c) {
                const size_t i = (size_t)m * 256 + c;
                float v;
                if (sp.lut_prec == FA_LUT_F32) {
                    memcpy(&v, raw.data() + 4 * i, 4);
                } else if (sp.lut_prec == FA_LUT_F16) {
                    uint16_t h;
                    memcpy(&h, raw.data() + 2 * i, 2);
                    v = half_bits_to_float(h) * sc[2 * m] + sc[2 * m + 1];
                } else {
                    v = e4m3_bits_to_float(raw[i]) * sc[2 * m] + sc[2 * m + 1];
                }
                out_lut[i] = v;
            }
    });
}

const char *fa_last_error(void) { return fa::last_error(); }

const char *fa_status_str(fa_status s) {
    switch (s) {
        case FA_OK: return "FA_OK";
        case FA_ERR_ARG: return "FA_ERR_ARG";
        case FA_ERR_OOM: return "FA_ERR_OOM";
        case FA_ERR_CUDA: return "FA_ERR_CUDA";
        case FA_ERR_TIMEOUT: return "FA_ERR_TIMEOUT";
        case FA_ERR_OVERFLOW: return "FA_ERR_OVERFLOW";
        case FA_ERR_STATE: return "FA_ERR_STATE";
        case FA_ERR_BUSY: return "FA_ERR_BUSY";
        case FA_ERR_IO: return "FA_ERR_IO";
        case FA_ERR_NODEV: return "FA_ERR_NODEV";
    }
    return "FA_ERR_UNKNOWN";
}

const char *fa_version(void) { return "fa 0.1 (sm_103a)"; }

}  // extern "C"
