// Offline index build (the offline processing of Section 3 and §4.1):
//   coarse k-means into nlist posting lists (Lloyd iterations on a sample),
//   Eq. 2 boundary replication (a vector joins every list C_i with
//     |v - C_i| <= (1 + eps) |v - C_1|, at most max_lists_per_vec lists),
//   PQ training (M sub-codebooks of 256 centroids over contiguous blocks of
//     d/M coordinates, §2.2) and encoding (nearest sub-centroid).
// The paper clusters with a hierarchical balanced algorithm and about 0.1*N
// lists; this build uses plain k-means with a given nlist. The assignment
// steps (k-means iterations over the sample, final nearest-r lists, encoding)
// run on the GPU kernels of this library when use_gpu is set and on host
// threads otherwise.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "fa_internal.h"

namespace fa {
namespace {

// lists from which the GPU build clusters in two levels
constexpr int32_t TWO_LEVEL_LISTS = 32768;

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the build's only random source.
struct SplitMix {
    uint64_t s;
    explicit SplitMix(uint64_t seed) : s(seed) {}
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
    uint64_t below(uint64_t m) { return next() % m; }
};

void row_f32(const void *base, fa_dtype dt, int32_t d, int64_t i, float *out) {
    if (dt == FA_F32) {
        memcpy(out, (const float *)base + i * d, sizeof(float) * d);
    } else if (dt == FA_I8) {
        const int8_t *p = (const int8_t *)base + i * d;
        for (int j = 0; j < d; ++j) out[j] = (float)p[j];
    } else {
        const uint8_t *p = (const uint8_t *)base + i * d;
        for (int j = 0; j < d; ++j) out[j] = (float)p[j];
    }
}

// nearest-r centroids of every row (host threads), squared L2 ascending
void host_assign_topr(const float *X, int64_t n, int32_t d, const float *C, int32_t K, int32_t r,
                      int32_t *ids, float *d2) {
#pragma omp parallel
    {
        std::vector<std::pair<float, int32_t>> best(r);
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) {
            const float *x = X + i * d;
            int cnt = 0;
            for (int32_t c = 0; c < K; ++c) {
                const float *cc = C + (int64_t)c * d;
                float s = 0.f;
                for (int j = 0; j < d; ++j) {
                    const float t = x[j] - cc[j];
                    s += t * t;
                }
                const std::pair<float, int32_t> cand{s, c};
                if (cnt < r) {
                    best[cnt++] = cand;
                    std::push_heap(best.begin(), best.begin() + cnt);
                } else if (cand < best[0]) {
                    std::pop_heap(best.begin(), best.begin() + cnt);
                    best[cnt - 1] = cand;
                    std::push_heap(best.begin(), best.begin() + cnt);
                }
            }
            std::sort_heap(best.begin(), best.begin() + cnt);
            for (int t = 0; t < r; ++t) {
                ids[i * r + t] = t < cnt ? best[t].second : -1;
                if (d2) d2[i * r + t] = t < cnt ? best[t].first : INFINITY;
            }
        }
    }
}

void assign1(const float *X, int64_t n, int32_t d, const float *C, int32_t K, bool gpu,
             int32_t *ids) {
    if (gpu)
        gpu_assign_topr(X, n, d, FA_F32, C, K, 1, ids, nullptr);
    else
        host_assign_topr(X, n, d, C, K, 1, ids, nullptr);
}

// Lloyd k-means on X[n][d] into K centroids; returns C[K][d].
std::vector<float> kmeans(const float *X, int64_t n, int32_t d, int32_t K, int iters,
                          uint64_t seed, bool gpu) {
    SplitMix rng(seed);
    std::vector<float> C((size_t)K * d);
    // initial centroids: K distinct sample rows (partial Fisher-Yates)
    std::vector<int64_t> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    for (int32_t c = 0; c < K; ++c) {
        const int64_t src = c < n ? c + (int64_t)rng.below((uint64_t)(n - c)) : (int64_t)rng.below(n);
        if (c < n) std::swap(idx[c], idx[src]);
        const int64_t row = c < n ? idx[c] : idx[src];
        memcpy(&C[(size_t)c * d], X + row * d, sizeof(float) * d);
        if (c >= n)  // more centroids than rows: jitter duplicates
            for (int j = 0; j < d; ++j) C[(size_t)c * d + j] += (float)(1e-3 * (rng.uniform() - 0.5));
    }
    std::vector<int32_t> a(n);
    std::vector<int64_t> count(K);
    std::vector<double> sum((size_t)K * d);
    for (int it = 0; it < iters; ++it) {
        assign1(X, n, d, C.data(), K, gpu, a.data());
        std::fill(count.begin(), count.end(), 0);
        for (int64_t i = 0; i < n; ++i) count[a[i]]++;
        // members of each cluster (counting sort), then per-cluster sums
        std::vector<int64_t> off(K + 1, 0), mem(n);
        for (int c = 0; c < K; ++c) off[c + 1] = off[c] + count[c];
        {
            std::vector<int64_t> fill(off.begin(), off.end() - 1);
            for (int64_t i = 0; i < n; ++i) mem[fill[a[i]]++] = i;
        }
#pragma omp parallel for schedule(dynamic, 16)
        for (int c = 0; c < K; ++c) {
            if (count[c] == 0) continue;
            double *s = &sum[(size_t)c * d];
            std::fill(s, s + d, 0.0);
            for (int64_t e = off[c]; e < off[c + 1]; ++e) {
                const float *x = X + mem[e] * d;
                for (int j = 0; j < d; ++j) s[j] += x[j];
            }
            for (int j = 0; j < d; ++j) C[(size_t)c * d + j] = (float)(s[j] / count[c]);
        }
        // empty clusters: split the largest cluster's centroid
        for (int c = 0; c < K; ++c) {
            if (count[c] > 0) continue;
            const int big = (int)(std::max_element(count.begin(), count.end()) - count.begin());
            for (int j = 0; j < d; ++j) {
                const float e = (float)(1e-4 * (rng.uniform() - 0.5)) * (1.f + fabsf(C[(size_t)big * d + j]));
                C[(size_t)c * d + j] = C[(size_t)big * d + j] + e;
                C[(size_t)big * d + j] -= e;
            }
            count[c] = count[big] / 2;
            count[big] -= count[c];
        }
    }
    return C;
}

// Two-level k-means for many lists (the paper clusters with a hierarchical
// balanced algorithm, §4.1): K1 ~ sqrt(nlist) top-level clusters by Lloyd
// k-means on a sub-sample, then each cluster's share of the nlist lists
// (proportional to its sample rows, largest remainder, at least one) by Lloyd
// k-means in which a row looks among the lists of its three nearest
// top-level clusters. Returns the list centroids grouped by
// top-level cluster: lists sub_beg[t] .. sub_beg[t + 1] - 1 belong to
// cluster t, whose centroid is top[t].
std::vector<float> kmeans_two_level(const float *X, int64_t n, int32_t d, int32_t nlist, int iters,
                                    uint64_t seed, std::vector<float> &top,
                                    std::vector<int32_t> &sub_beg) {
    int32_t K1 = (int32_t)llround(sqrt((double)nlist));
    K1 = std::max(2, std::min(K1, std::min<int32_t>(nlist, 2048)));
    const int64_t S1 = std::min<int64_t>(n, 256ll * K1);
    std::vector<float> X1((size_t)S1 * d);
    for (int64_t i = 0; i < S1; ++i) memcpy(&X1[(size_t)i * d], X + ((i * n) / S1) * d, sizeof(float) * d);
    top = kmeans(X1.data(), S1, d, K1, iters, seed ^ 0x746f70ull, true);

    // the sample's top-level clusters and each cluster's list count
    std::vector<int32_t> cl(n);
    gpu_assign_topr(X, n, d, FA_F32, top.data(), K1, 1, cl.data(), nullptr);
    std::vector<int64_t> cnt(K1, 0);
    for (int64_t i = 0; i < n; ++i) cnt[cl[i]]++;
    std::vector<int32_t> K2(K1, 1);
    {
        const int64_t spare = nlist - K1;  // one list each, then the rest by rows
        std::vector<std::pair<double, int32_t>> frac(K1);
        int64_t given = 0;
        for (int t = 0; t < K1; ++t) {
            const double share = (double)spare * (double)cnt[t] / (double)n;
            const int64_t f = (int64_t)share;
            K2[t] += (int32_t)f;
            given += f;
            frac[t] = {share - (double)f, t};
        }
        std::sort(frac.begin(), frac.end(), [](const std::pair<double, int32_t> &a,
                                               const std::pair<double, int32_t> &b) {
            return a.first != b.first ? a.first > b.first : a.second < b.second;
        });
        for (int64_t i = 0; i < spare - given; ++i) K2[frac[(size_t)(i % K1)].second]++;
    }
    sub_beg.assign(K1 + 1, 0);
    for (int t = 0; t < K1; ++t) sub_beg[t + 1] = sub_beg[t] + K2[t];

    // members of each cluster, then the initial lists: evenly spaced members
    std::vector<int64_t> off(K1 + 1, 0), mem(n);
    for (int t = 0; t < K1; ++t) off[t + 1] = off[t] + cnt[t];
    {
        std::vector<int64_t> fill(off.begin(), off.end() - 1);
        for (int64_t i = 0; i < n; ++i) mem[fill[cl[i]]++] = i;
    }
    std::vector<float> C((size_t)nlist * d);
    SplitMix rng(seed ^ 0x7375626cull);
    for (int t = 0; t < K1; ++t)
        for (int32_t j = 0; j < K2[t]; ++j) {
            float *c = &C[(size_t)(sub_beg[t] + j) * d];
            if (cnt[t] > 0) {
                memcpy(c, X + mem[off[t] + (j * cnt[t]) / K2[t]] * d, sizeof(float) * d);
                if (j >= cnt[t])  // more lists than rows: jitter the repeats
                    for (int k = 0; k < d; ++k) c[k] += (float)(1e-3 * (rng.uniform() - 0.5));
            } else {
                memcpy(c, &top[(size_t)t * d], sizeof(float) * d);
            }
        }
    std::vector<int32_t> a(n);
    std::vector<int64_t> lc(nlist);
    std::vector<double> sum((size_t)nlist * d);
    for (int it = 0; it < iters; ++it) {
        gpu_assign_two_level(X, n, d, FA_F32, top.data(), K1, C.data(), nlist, sub_beg.data(), 1,
                             a.data(), nullptr, nullptr);
        std::fill(lc.begin(), lc.end(), 0);
        std::fill(sum.begin(), sum.end(), 0.0);
        for (int64_t i = 0; i < n; ++i) {
            const int32_t l = a[i];
            if (l < 0) continue;
            lc[l]++;
            double *sl = &sum[(size_t)l * d];
            const float *x = X + i * d;
            for (int k = 0; k < d; ++k) sl[k] += x[k];
        }
#pragma omp parallel for schedule(static)
        for (int32_t l = 0; l < nlist; ++l)
            if (lc[l] > 0)
                for (int k = 0; k < d; ++k) C[(size_t)l * d + k] = (float)(sum[(size_t)l * d + k] / lc[l]);
        // an empty list splits the largest list of its cluster
        for (int t = 0; t < K1; ++t)
            for (int32_t l = sub_beg[t]; l < sub_beg[t + 1]; ++l) {
                if (lc[l] > 0) continue;
                int32_t big = sub_beg[t];
                for (int32_t m = sub_beg[t]; m < sub_beg[t + 1]; ++m)
                    if (lc[m] > lc[big]) big = m;
                if (lc[big] < 2) continue;
                for (int k = 0; k < d; ++k) {
                    const float e = (float)(1e-4 * (rng.uniform() - 0.5)) * (1.f + fabsf(C[(size_t)big * d + k]));
                    C[(size_t)l * d + k] = C[(size_t)big * d + k] + e;
                    C[(size_t)big * d + k] -= e;
                }
                lc[l] = lc[big] / 2;
                lc[big] -= lc[l];
            }
    }
    return C;
}

void host_encode(const void *base, int64_t n, int32_t d, fa_dtype dt, const float *cb, int32_t M,
                 uint8_t *codes) {
    const int dsub = d / M;
#pragma omp parallel
    {
        std::vector<float> x(d);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            row_f32(base, dt, d, i, x.data());
            for (int m = 0; m < M; ++m) {
                float best = INFINITY;
                int bc = 0;
                for (int c = 0; c < 256; ++c) {
                    const float *w = cb + ((int64_t)m * 256 + c) * dsub;
                    float s = 0.f;
                    for (int j = 0; j < dsub; ++j) {
                        const float t = x[m * dsub + j] - w[j];
                        s += t * t;
                    }
                    if (s < best) {
                        best = s;
                        bc = c;
                    }
                }
                codes[i * M + m] = (uint8_t)bc;
            }
        }
    }
}

}  // namespace

void train_and_encode(const void *base, int64_t n, int32_t d, fa_dtype dt,
                      const fa_build_params &p, BuildOut &out) {
    const int32_t nlist = p.nlist, M = p.M, dsub = d / M;
    const bool gpu = p.use_gpu != 0;
    const int iters = p.kmeans_iters;
    // many lists on the GPU: two-level clustering (hierarchical, §4.1), with
    // each vector's lists found inside its top-level cluster
    const bool two_level = gpu && nlist >= TWO_LEVEL_LISTS;
    // training sample: evenly strided rows
    int64_t S = p.train_sample > 0 ? std::min<int64_t>(n, p.train_sample)
                                   : std::min<int64_t>(n, std::max<int64_t>(65536, (two_level ? 24ll : 64ll) * nlist));
    std::vector<float> X((size_t)S * d);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < S; ++i) row_f32(base, dt, d, (i * n) / S, &X[(size_t)i * d]);

    // coarse quantizer
    std::vector<float> top;
    std::vector<int32_t> sub_beg;
    if (two_level)
        out.centroids = kmeans_two_level(X.data(), S, d, nlist, iters, p.seed ^ 0x636f61727365ull, top, sub_beg);
    else
        out.centroids = kmeans(X.data(), S, d, nlist, iters, p.seed ^ 0x636f61727365ull, gpu);

    // assignment with Eq. 2 replication
    const int32_t r = p.repl_eps != 0.f ? p.max_lists_per_vec : 1;
    std::vector<int32_t> ids((size_t)n * r);
    std::vector<float> d2((size_t)n * r);
    if (two_level) {
        gpu_assign_two_level(base, n, d, dt, top.data(), (int32_t)top.size() / d, out.centroids.data(),
                             nlist, sub_beg.data(), r, ids.data(), d2.data(), nullptr);
    } else if (gpu) {
        gpu_assign_topr(base, n, d, dt, out.centroids.data(), nlist, r, ids.data(), d2.data());
    } else {
        const int64_t chunk = 1 << 16;
        std::vector<float> xb((size_t)chunk * d);
        for (int64_t r0 = 0; r0 < n; r0 += chunk) {
            const int64_t cnt = std::min(chunk, n - r0);
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < cnt; ++i) row_f32(base, dt, d, r0 + i, &xb[(size_t)i * d]);
            host_assign_topr(xb.data(), cnt, d, out.centroids.data(), nlist, r, &ids[(size_t)r0 * r],
                             &d2[(size_t)r0 * r]);
        }
    }
    // Eq. 2's epsilon: given, or (repl_eps < 0) chosen by bisection so that a
    // vector joins -repl_eps lists on average, measured on up to 1M vectors
    // drawn by a multiplicative hash of the row index: a strided sample would
    // line up with the k-means training rows, which sit closer to the centroids
    // fitted to them and join fewer lists than the rest
    double eps = p.repl_eps;
    if (p.repl_eps < 0.f && r > 1) {
        const double target = -(double)p.repl_eps;
        const int64_t ns = std::min<int64_t>(n, 1 << 20);
        auto mean_lists = [&](double e) {
            int64_t tot = 0;
#pragma omp parallel for reduction(+ : tot) schedule(static)
            for (int64_t s2 = 0; s2 < ns; ++s2) {
                const int64_t i = ns == n ? s2 : (int64_t)(((uint64_t)s2 * 2654435761ull) % (uint64_t)n);
                const double lim = (1.0 + e) * sqrt((double)std::max(0.f, d2[(size_t)i * r]));
                int c = 1;
                for (int t = 1; t < r; ++t) {
                    if (ids[(size_t)i * r + t] < 0) break;
                    if (sqrt((double)std::max(0.f, d2[(size_t)i * r + t])) <= lim) ++c;
                    else break;
                }
                tot += c;
            }
            return (double)tot / (double)ns;
        };
        double lo = 0.0, hi = 1.0;
        while (hi < 64.0 && mean_lists(hi) < target) hi *= 2.0;
        for (int it = 0; it < 40; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mean_lists(mid) < target) lo = mid;
            else hi = mid;
        }
        eps = hi;
    }
    out.repl_eps = (float)eps;
    out.primary.resize(n);
    std::vector<std::vector<int64_t>> rep(nlist);
    for (int64_t i = 0; i < n; ++i) {
        out.primary[i] = ids[(size_t)i * r];
        const double lim = (1.0 + eps) * sqrt((double)std::max(0.f, d2[(size_t)i * r]));
        for (int t = 1; t < r; ++t) {
            const int32_t l = ids[(size_t)i * r + t];
            if (l < 0) break;
            if (sqrt((double)std::max(0.f, d2[(size_t)i * r + t])) <= lim) rep[l].push_back(i);
            else break;  // candidates are ascending: the rest are farther
        }
    }
    out.rep_off.assign(nlist + 1, 0);
    for (int l = 0; l < nlist; ++l) out.rep_off[l + 1] = out.rep_off[l] + (int64_t)rep[l].size();
    out.rep_ids.clear();
    out.rep_ids.reserve(out.rep_off[nlist]);
    for (int l = 0; l < nlist; ++l) out.rep_ids.insert(out.rep_ids.end(), rep[l].begin(), rep[l].end());

    train_pq_and_encode(base, n, d, dt, p, X.data(), S, out);
}

// PQ sub-codebooks (one k-means per subspace on a sub-sample of the training
// rows X[S][d]) and the code of every base vector.
void train_pq_and_encode(const void *base, int64_t n, int32_t d, fa_dtype dt,
                         const fa_build_params &p, const float *X, int64_t S, BuildOut &out) {
    const int32_t M = p.M, dsub = d / M;
    const bool gpu = p.use_gpu != 0;
    const int iters = p.kmeans_iters;
    const int64_t Sp = std::min<int64_t>(S, 32768);
    out.codebooks.assign((size_t)M * 256 * dsub, 0.f);
#pragma omp parallel for schedule(dynamic, 1)
    for (int m = 0; m < M; ++m) {
        std::vector<float> sub((size_t)Sp * dsub);
        for (int64_t i = 0; i < Sp; ++i)
            memcpy(&sub[(size_t)i * dsub], &X[(size_t)((i * S) / Sp) * d + m * dsub], sizeof(float) * dsub);
        std::vector<float> cb =
            kmeans(sub.data(), Sp, dsub, 256, iters, p.seed ^ (0x7071ull << 16) ^ (uint64_t)m, false);
        memcpy(&out.codebooks[(size_t)m * 256 * dsub], cb.data(), sizeof(float) * 256 * dsub);
    }

    out.codes.resize((size_t)n * M);
    if (gpu)
        gpu_encode(base, n, d, dt, out.codebooks.data(), M, out.codes.data());
    else
        host_encode(base, n, d, dt, out.codebooks.data(), M, out.codes.data());
}

// Lists given by the caller (centroids and the list of every vector): only the
// PQ part is trained.
void encode_with_lists(const void *base, int64_t n, int32_t d, fa_dtype dt,
                       const fa_build_params &p, BuildOut &out) {
    const int64_t S = p.train_sample > 0 ? std::min<int64_t>(n, p.train_sample)
                                         : std::min<int64_t>(n, 65536);
    std::vector<float> X((size_t)S * d);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < S; ++i) row_f32(base, dt, d, (i * n) / S, &X[(size_t)i * d]);
    train_pq_and_encode(base, n, d, dt, p, X.data(), S, out);
}

// Storage layout of the raw vectors on the slow tier (§4.3): the vectors
// whose primary list is l form bucket l (ascending ids), a page holds cap
// of them. Every bucket fills whole pages of its own first (pages numbered by
// list); the rest of each bucket (a tail shorter than a page) is packed into
// shared pages by a max-min rule: the largest unplaced tail opens a page and
// the smallest unplaced tails join it, smallest first, while they fit (ties
// by list). Returns the page count.
int64_t page_layout(const std::vector<int32_t> &primary, int32_t nlist, int32_t cap,
                    std::vector<int64_t> &page_of, std::vector<int32_t> &slot_of) {
    const int64_t n = (int64_t)primary.size();
    std::vector<std::vector<int64_t>> bucket(nlist);
    for (int64_t v = 0; v < n; ++v) bucket[primary[v]].push_back(v);
    page_of.assign(n, -1);
    slot_of.assign(n, -1);
    int64_t page = 0;
    std::vector<std::pair<int64_t, int32_t>> tails;  // (size, list)
    for (int32_t l = 0; l < nlist; ++l) {
        const std::vector<int64_t> &b = bucket[l];
        const int64_t whole = (int64_t)b.size() / cap;
        for (int64_t t = 0; t < whole * cap; ++t) {
            page_of[b[t]] = page + t / cap;
            slot_of[b[t]] = (int32_t)(t % cap);
        }
        page += whole;
        if (b.size() % cap) tails.push_back({(int64_t)(b.size() % cap), l});
    }
    std::sort(tails.begin(), tails.end(), [](const std::pair<int64_t, int32_t> &a,
                                             const std::pair<int64_t, int32_t> &b) {
        return a.first != b.first ? a.first > b.first : a.second < b.second;
    });
    std::vector<char> placed(tails.size(), 0);
    int64_t lo = (int64_t)tails.size() - 1;
    for (size_t hi = 0; hi < tails.size(); ++hi) {
        if (placed[hi]) continue;
        int64_t room = cap, slot = 0;
        size_t pick = hi;
        for (;;) {
            const std::vector<int64_t> &b = bucket[tails[pick].second];
            const int64_t sz = tails[pick].first, from = (int64_t)b.size() - sz;
            for (int64_t t = 0; t < sz; ++t) {
                page_of[b[from + t]] = page;
                slot_of[b[from + t]] = (int32_t)(slot + t);
            }
            slot += sz;
            room -= sz;
            placed[pick] = 1;
            while (lo > (int64_t)hi && placed[lo]) --lo;
            if (lo <= (int64_t)hi || tails[lo].first > room) break;
            pick = (size_t)lo;
        }
        ++page;
    }
    return page;
}

}  // namespace fa
