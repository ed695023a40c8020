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
    if (dt == FA_F32)
        memcpy(out, (const float *)base + i * d, sizeof(float) * d);
    else {
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
    // training sample: evenly strided rows
    int64_t S = p.train_sample > 0 ? std::min<int64_t>(n, p.train_sample)
                                   : std::min<int64_t>(n, std::max<int64_t>(65536, 64ll * nlist));
    std::vector<float> X((size_t)S * d);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < S; ++i) row_f32(base, dt, d, (i * n) / S, &X[(size_t)i * d]);

    // coarse quantizer
    out.centroids = kmeans(X.data(), S, d, nlist, iters, p.seed ^ 0x636f61727365ull, gpu);

    // assignment with Eq. 2 replication
    const int32_t r = p.repl_eps > 0.f ? p.max_lists_per_vec : 1;
    std::vector<int32_t> ids((size_t)n * r);
    std::vector<float> d2((size_t)n * r);
    if (gpu) {
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
    out.primary.resize(n);
    std::vector<std::vector<int64_t>> rep(nlist);
    for (int64_t i = 0; i < n; ++i) {
        out.primary[i] = ids[(size_t)i * r];
        const double lim = (1.0 + (double)p.repl_eps) * sqrt((double)std::max(0.f, d2[(size_t)i * r]));
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

}  // namespace fa
