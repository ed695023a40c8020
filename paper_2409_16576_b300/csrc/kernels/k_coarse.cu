// Step 2 of the filtering path (coarse probe): the nprobe posting lists whose
// centroids are nearest to each query. The paper walks an SPTAG graph on the
// CPU (§4.1 "In-memory Indices"); here the exact top-nprobe is computed on the
// GPU. This file holds the FP32 direct-difference form:
//   k_l2_tile   squared L2 between a tile of rows and a tile of centroids
//               (FP32, sum of (x_j - c_j)^2, no cancellation)
//   k_select    per-row top-n of those distances by (distance, column)
// The same two kernels serve the GPU-assisted index build (nearest-r lists of
// every base vector for Eq. 2, k-means assignment). k_encode picks the PQ
// code of every subspace (nearest of the 256 sub-centroids).
#include <algorithm>
#include <mutex>
#include <string>

#include "../fa_internal.h"
#include "warp_topk.cuh"

namespace fa {

constexpr int TILE = 64;
constexpr int KC = 32;  // dimensions per smem stage
constexpr int LDS = TILE + 4;

// ip != 0: the negated inner product -<x, c> instead of the squared L2.
__global__ void __launch_bounds__(256) k_l2_tile(const float *__restrict__ X, int64_t nx,
                                                 const float *__restrict__ C, int32_t nc,
                                                 int32_t d, float *__restrict__ D, int64_t ldd, int ip) {
    __shared__ __align__(16) float xs[KC][LDS];
    __shared__ __align__(16) float cs[KC][LDS];
    const int t = threadIdx.x;
    const int ty = t >> 4, tx = t & 15;
    const int64_t row0 = (int64_t)blockIdx.y * TILE;
    const int64_t col0 = (int64_t)blockIdx.x * TILE;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    for (int k0 = 0; k0 < d; k0 += KC) {
        // stage a 64 x 32 slice of rows and of centroids, transposed
        for (int e = t; e < TILE * KC; e += 256) {
            const int r = e / KC, k = e % KC;
            const int64_t xr = row0 + r, cr = col0 + r;
            const int kk = k0 + k;
            xs[k][r] = (xr < nx && kk < d) ? X[xr * d + kk] : 0.f;
            cs[k][r] = (cr < nc && kk < d) ? C[cr * d + kk] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < KC; ++k) {
            const float4 a = *reinterpret_cast<const float4 *>(&xs[k][ty * 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&cs[k][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (ip) {
                        acc[i][j] = fmaf(-av[i], bv[j], acc[i][j]);
                    } else {
                        const float df = av[i] - bv[j];
                        acc[i][j] = fmaf(df, df, acc[i][j]);
                    }
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t r = row0 + ty * 4 + i;
        if (r >= nx) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t c = col0 + tx * 4 + j;
            if (c < nc) D[r * ldd + c] = acc[i][j];
        }
    }
}

template <int R>
__global__ void __launch_bounds__(256) k_select(const float *__restrict__ D, int64_t ldd,
                                                int64_t nrows, int32_t nc, int32_t ntop,
                                                int32_t *__restrict__ out_ids, int32_t out_stride,
                                                float *__restrict__ out_d2) {
    __shared__ uint64_t wbuf[8][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * 8 + warp;
    if (row >= nrows) return;
    WarpTopK<R> tk;
    tk.init(wbuf[warp], ntop);
    const float *dr = D + row * ldd;
    for (int c0 = 0; c0 < nc; c0 += 32) {
        const int c = c0 + lane;
        const bool ok = c < nc;
        const float v = ok ? dr[c] : 0.f;
        tk.push(make_key(v, (uint32_t)c), ok);
    }
    tk.finish();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = r * 32 + lane;
        if (e < ntop) {
            const uint64_t k = tk.L[r];
            out_ids[row * out_stride + e] = k == KEY_INF ? -1 : (int32_t)(k & 0xffffffffu);
            if (out_d2) out_d2[row * out_stride + e] = k == KEY_INF ? INFINITY : o2f((uint32_t)(k >> 32));
        }
    }
}

static void select_rows(const float *D, int64_t ldd, int64_t nrows, int32_t nc, int32_t ntop,
                        int32_t *out_ids, int32_t out_stride, float *out_d2, cudaStream_t st) {
    const dim3 grid((unsigned)((nrows + 7) / 8));
    if (ntop <= 32)
        k_select<1><<<grid, 256, 0, st>>>(D, ldd, nrows, nc, ntop, out_ids, out_stride, out_d2);
    else if (ntop <= 64)
        k_select<2><<<grid, 256, 0, st>>>(D, ldd, nrows, nc, ntop, out_ids, out_stride, out_d2);
    else if (ntop <= 128)
        k_select<4><<<grid, 256, 0, st>>>(D, ldd, nrows, nc, ntop, out_ids, out_stride, out_d2);
    else if (ntop <= 256)
        k_select<8><<<grid, 256, 0, st>>>(D, ldd, nrows, nc, ntop, out_ids, out_stride, out_d2);
    else if (ntop <= 512)
        k_select<16><<<grid, 256, 0, st>>>(D, ldd, nrows, nc, ntop, out_ids, out_stride, out_d2);
    else
        FA_REQUIRE(false, FA_ERR_ARG, "top-n of the coarse probe above 512");
    FA_CHECK_CUDA(cudaGetLastError());
}

// rows x centroids -> top-ntop columns per row, in blocks of rows so that the
// distance scratch stays within the workspace's coarse buffer.
static void l2_topn(const float *X, int64_t nx, int32_t d, const float *C, int32_t nc,
                    int32_t ntop, float *scratch, int64_t scratch_rows, int32_t *out_ids,
                    int32_t out_stride, float *out_d2, cudaStream_t st, int ip = 0) {
    // a block of rows spans at most 65535 tiles in y (the grid's y limit)
    if (scratch_rows > (int64_t)65535 * TILE) scratch_rows = (int64_t)65535 * TILE;
    for (int64_t r0 = 0; r0 < nx; r0 += scratch_rows) {
        const int64_t rows = nx - r0 < scratch_rows ? nx - r0 : scratch_rows;
        const dim3 grid((unsigned)((nc + TILE - 1) / TILE), (unsigned)((rows + TILE - 1) / TILE));
        k_l2_tile<<<grid, 256, 0, st>>>(X + r0 * d, rows, C, nc, d, scratch, nc, ip);
        FA_CHECK_CUDA(cudaGetLastError());
        select_rows(scratch, nc, rows, nc, ntop, out_ids + r0 * out_stride, out_stride,
                    out_d2 ? out_d2 + r0 * out_stride : nullptr, st);
    }
}

void launch_l2_topn(const float *X, int64_t nx, int32_t d, const float *C, int32_t nc, int32_t ntop,
                    float *scratch, int64_t scratch_rows, int32_t *out_ids, int32_t out_stride,
                    cudaStream_t st, int ip) {
    l2_topn(X, nx, d, C, nc, ntop, scratch, scratch_rows, out_ids, out_stride, nullptr, st, ip);
}

void launch_coarse(const DeviceIndex &ix, const float *q, int64_t nq, int32_t nprobe,
                   int32_t probe_stride, int gemm, Workspace &ws, int32_t *probes,
                   cudaStream_t st) {
    if (nq == 0) return;
    if (gemm == FA_GEMM_BF16_TC && ix.centroids_bf16) {
        // distances on the tensor cores, then the per-row top-nprobe
        for (int64_t r0 = 0; r0 < nq; r0 += ws.coarse_rows) {
            const int64_t rows = std::min(ws.coarse_rows, nq - r0);
            launch_coarse_tc(ix, q + r0 * ix.d, rows, nprobe, ws.coarse_d, probes + r0 * probe_stride,
                             probe_stride, ws.err, st);
        }
        return;
    }
    l2_topn(q, nq, ix.d, ix.centroids, ix.nlist, nprobe, ws.coarse_d, ws.coarse_rows, probes,
            probe_stride, nullptr, st, ix.metric == FA_METRIC_IP ? 1 : 0);
}

int coarse_launches(const DeviceIndex &ix, int64_t nq, int gemm, const Workspace &ws) {
    if (nq == 0) return 0;
    (void)gemm;
    return (int)(2 * ((nq + ws.coarse_rows - 1) / ws.coarse_rows));
}

// ---------------------------------------------------------------------------
// build helpers
// ---------------------------------------------------------------------------
__global__ void k_u8_to_f32(const uint8_t *__restrict__ src, float *__restrict__ dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

__global__ void k_i8_to_f32(const int8_t *__restrict__ src, float *__restrict__ dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

__global__ void k_encode(const float *__restrict__ X, int64_t n, int32_t d,
                         const float *__restrict__ cb, int32_t M, uint8_t *__restrict__ codes) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * M) return;
    const int64_t row = idx / M;
    const int m = (int)(idx - row * M);
    const int dsub = d / M;
    const float *x = X + row * d + m * dsub;
    float xv[16];
    for (int j = 0; j < dsub; ++j) xv[j] = x[j];
    float best = INFINITY;
    int bc = 0;
    for (int c = 0; c < 256; ++c) {
        const float *w = cb + ((int64_t)m * 256 + c) * dsub;
        float s = 0.f;
        for (int j = 0; j < dsub; ++j) {
            const float t = xv[j] - w[j];
            s = fmaf(t, t, s);
        }
        if (s < best) {
            best = s;
            bc = c;
        }
    }
    codes[idx] = (uint8_t)bc;
}

// Fused distances and per-row top-r (r <= 8) for the index build: a CTA
// takes 64 rows and walks the columns in 64 x 64 tiles (the direct-difference
// tiles of k_l2_tile), and 64 of its threads fold each tile into their row's
// running top-8 kept in registers, so no distance matrix is written. Rows may
// come through an order (position p holds row xrow[p]) with a column range per
// position [cbeg[p], cend[p]) (the lists of the row's top-level cluster in the
// two-level build); the CTA walks the union of its rows' ranges and masks the
// rest. Ties go to the smaller column.
constexpr int TOPR_MAX = 8;

__global__ void __launch_bounds__(256) k_l2_topr(const float *__restrict__ X,
                                                 const int32_t *__restrict__ xrow, int64_t nx,
                                                 int32_t d, const float *__restrict__ C, int32_t nc,
                                                 const int32_t *__restrict__ cbeg,
                                                 const int32_t *__restrict__ cend, int32_t r,
                                                 int32_t *__restrict__ out_ids,
                                                 float *__restrict__ out_d2) {
    __shared__ __align__(16) float xs[KC][LDS];
    __shared__ __align__(16) float cs[KC][LDS];
    __shared__ float dt[TILE][TILE + 1];
    __shared__ int64_t s_row[TILE];
    __shared__ int32_t s_b[TILE], s_e[TILE];
    __shared__ int32_t s_lo, s_hi;
    const int t = threadIdx.x;
    const int ty = t >> 4, tx = t & 15;
    const int64_t p0 = (int64_t)blockIdx.x * TILE;
    if (t < TILE) {
        const int64_t p = p0 + t;
        const bool ok = p < nx;
        s_row[t] = ok ? (xrow ? (int64_t)xrow[p] : p) : -1;
        s_b[t] = ok ? (cbeg ? cbeg[p] : 0) : nc;
        s_e[t] = ok ? (cend ? cend[p] : nc) : 0;
    }
    if (t == 0) {
        s_lo = nc;
        s_hi = 0;
    }
    __syncthreads();
    if (t < TILE && s_row[t] >= 0) {
        atomicMin(&s_lo, s_b[t]);
        atomicMax(&s_hi, s_e[t]);
    }
    __syncthreads();
    const int lo = s_lo, hi = s_hi;
    float bd[TOPR_MAX];
    int32_t bi[TOPR_MAX];
#pragma unroll
    for (int i = 0; i < TOPR_MAX; ++i) {
        bd[i] = INFINITY;
        bi[i] = -1;
    }
    for (int c0 = lo - lo % TILE; c0 < hi; c0 += TILE) {
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        for (int k0 = 0; k0 < d; k0 += KC) {
            for (int e = t; e < TILE * KC; e += 256) {
                const int rr = e / KC, k = e % KC;
                const int64_t xr = s_row[rr];
                const int64_t cr = (int64_t)c0 + rr;
                const int kk = k0 + k;
                xs[k][rr] = (xr >= 0 && kk < d) ? X[xr * d + kk] : 0.f;
                cs[k][rr] = (cr < nc && kk < d) ? C[cr * d + kk] : 0.f;
            }
            __syncthreads();
#pragma unroll 8
            for (int k = 0; k < KC; ++k) {
                const float4 a = *reinterpret_cast<const float4 *>(&xs[k][ty * 4]);
                const float4 b = *reinterpret_cast<const float4 *>(&cs[k][tx * 4]);
                const float av[4] = {a.x, a.y, a.z, a.w};
                const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float df = av[i] - bv[j];
                        acc[i][j] = fmaf(df, df, acc[i][j]);
                    }
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int rr = ty * 4 + i;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = c0 + tx * 4 + j;
                dt[rr][tx * 4 + j] = (c < nc && c >= s_b[rr] && c < s_e[rr]) ? acc[i][j] : INFINITY;
            }
        }
        __syncthreads();
        if (t < TILE) {
            for (int j = 0; j < TILE; ++j) {
                float cv = dt[t][j];
                if (!(cv < bd[TOPR_MAX - 1])) continue;
                int32_t ci = c0 + j;
#pragma unroll
                for (int s2 = 0; s2 < TOPR_MAX; ++s2)
                    if (cv < bd[s2]) {
                        const float tv = bd[s2];
                        const int32_t ti = bi[s2];
                        bd[s2] = cv;
                        bi[s2] = ci;
                        cv = tv;
                        ci = ti;
                    }
            }
        }
        __syncthreads();
    }
    if (t < TILE && s_row[t] >= 0) {
        const int64_t row = s_row[t];
#pragma unroll
        for (int i = 0; i < TOPR_MAX; ++i)
            if (i < r) {
                out_ids[row * r + i] = bi[i];
                if (out_d2) out_d2[row * r + i] = bd[i];
            }
    }
}

// Column range of each position of a two-level assignment: the lists of the
// position's row's j-th nearest top-level cluster (sup has `stride` clusters a row).
__global__ void k_seg_ranges(const int32_t *__restrict__ order, const int32_t *__restrict__ sup,
                             int32_t stride, int64_t n, const int32_t *__restrict__ sub_beg,
                             int32_t nsup, int32_t *__restrict__ cbeg, int32_t *__restrict__ cend) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s2 = sup[(int64_t)order[p] * stride];
        const bool ok = s2 >= 0 && s2 < nsup;
        cbeg[p] = ok ? sub_beg[s2] : 0;
        cend[p] = ok ? sub_beg[s2 + 1] : 0;
    }
}

// Per row, the r smallest (distance, list) pairs of two ascending lists of r
// (the running lists a and one more cluster's b); a keeps the result.
__global__ void k_merge_topr(int32_t *__restrict__ ai, float *__restrict__ ad,
                             const int32_t *__restrict__ bi, const float *__restrict__ bd, int64_t n,
                             int32_t r) {
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
         row += (int64_t)gridDim.x * blockDim.x) {
        int32_t oi[TOPR_MAX];
        float od[TOPR_MAX];
        int x = 0, y = 0;
        for (int t = 0; t < r; ++t) {
            const float da = x < r ? ad[row * r + x] : INFINITY;
            const float db = y < r ? bd[row * r + y] : INFINITY;
            const int32_t ia = x < r ? ai[row * r + x] : -1;
            const int32_t ib = y < r ? bi[row * r + y] : -1;
            const bool take_a = ib < 0 || (ia >= 0 && (da < db || (da == db && ia < ib)));
            if (take_a) {
                oi[t] = ia;
                od[t] = da;
                ++x;
            } else {
                oi[t] = ib;
                od[t] = db;
                ++y;
            }
        }
        for (int t = 0; t < r; ++t) {
            ai[row * r + t] = oi[t];
            ad[row * r + t] = od[t];
        }
    }
}

namespace {
struct DevBuf {
    void *p = nullptr;
    explicit DevBuf(size_t bytes) { FA_CHECK_CUDA(cudaMalloc(&p, bytes ? bytes : 1)); }
    ~DevBuf() { cudaFree(p); }
    template <class T> T *as() { return reinterpret_cast<T *>(p); }
};
}  // namespace

static void rows_to_f32(const void *rows, int64_t r0, int64_t cnt, int32_t d, fa_dtype dt,
                        float *dst, uint8_t *stage, cudaStream_t st) {
    if (dt == FA_F32) {
        FA_CHECK_CUDA(cudaMemcpyAsync(dst, (const float *)rows + r0 * d, sizeof(float) * cnt * d,
                                      cudaMemcpyHostToDevice, st));
    } else {
        FA_CHECK_CUDA(cudaMemcpyAsync(stage, (const uint8_t *)rows + r0 * d, (size_t)cnt * d,
                                      cudaMemcpyHostToDevice, st));
        if (dt == FA_I8)
            k_i8_to_f32<<<1024, 256, 0, st>>>(reinterpret_cast<const int8_t *>(stage), dst, cnt * d);
        else
            k_u8_to_f32<<<1024, 256, 0, st>>>(stage, dst, cnt * d);
        FA_CHECK_CUDA(cudaGetLastError());
    }
}

void gpu_assign_topr(const void *rows, int64_t n, int32_t d, fa_dtype dt, const float *centroids,
                     int32_t nlist, int32_t r, int32_t *out_ids, float *out_d2) {
    cudaStream_t st;
    FA_CHECK_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    const int64_t chunk = 1 << 20;
    const bool fused = r <= TOPR_MAX;
    const int64_t srows = fused ? 64 : std::max<int64_t>(64, std::min<int64_t>(chunk, (256ll << 20) / (4ll * nlist)));
    DevBuf dc(sizeof(float) * (size_t)nlist * d), dx(sizeof(float) * chunk * d),
        ds((size_t)chunk * d), dd(fused ? 4 : sizeof(float) * srows * nlist),
        di(sizeof(int32_t) * chunk * r), dd2(sizeof(float) * chunk * r);
    FA_CHECK_CUDA(cudaMemcpyAsync(dc.p, centroids, sizeof(float) * (size_t)nlist * d,
                                  cudaMemcpyHostToDevice, st));
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t cnt = std::min(chunk, n - r0);
        rows_to_f32(rows, r0, cnt, d, dt, dx.as<float>(), ds.as<uint8_t>(), st);
        if (fused) {
            k_l2_topr<<<(unsigned)((cnt + TILE - 1) / TILE), 256, 0, st>>>(
                dx.as<float>(), nullptr, cnt, d, dc.as<float>(), nlist, nullptr, nullptr, r,
                di.as<int32_t>(), dd2.as<float>());
            FA_CHECK_CUDA(cudaGetLastError());
        } else {
            l2_topn(dx.as<float>(), cnt, d, dc.as<float>(), nlist, r, dd.as<float>(), srows,
                    di.as<int32_t>(), r, dd2.as<float>(), st);
        }
        FA_CHECK_CUDA(cudaMemcpyAsync(out_ids + r0 * r, di.p, sizeof(int32_t) * cnt * r,
                                      cudaMemcpyDeviceToHost, st));
        if (out_d2)
            FA_CHECK_CUDA(cudaMemcpyAsync(out_d2 + r0 * r, dd2.p, sizeof(float) * cnt * r,
                                          cudaMemcpyDeviceToHost, st));
        FA_CHECK_CUDA(cudaStreamSynchronize(st));
    }
    cudaStreamDestroy(st);
}

void gpu_assign_two_level(const void *rows, int64_t n, int32_t d, fa_dtype dt, const float *top,
                          int32_t ntop, const float *lists, int32_t nlist, const int32_t *sub_beg,
                          int32_t r, int32_t *out_ids, float *out_d2, int32_t *out_top) {
    FA_REQUIRE(r >= 1 && r <= TOPR_MAX, FA_ERR_ARG, "two-level assignment keeps at most 8 lists");
    // the lists of a row's TP nearest top-level clusters are searched
    const int32_t TP = std::min<int32_t>(3, ntop);
    cudaStream_t st;
    FA_CHECK_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    const int64_t chunk = 1 << 20;
    DevBuf dtop(sizeof(float) * (size_t)ntop * d), dl(sizeof(float) * (size_t)nlist * d),
        dsb(sizeof(int32_t) * ((size_t)ntop + 1)), dx(sizeof(float) * chunk * d), ds((size_t)chunk * d),
        dsup(sizeof(int32_t) * chunk * TP), dcnt(sizeof(uint32_t) * (size_t)ntop), dord(sizeof(int32_t) * chunk),
        dcb(sizeof(int32_t) * chunk), dce(sizeof(int32_t) * chunk), di(sizeof(int32_t) * chunk * r),
        dd2(sizeof(float) * chunk * r), dj(sizeof(int32_t) * chunk * r), ddj(sizeof(float) * chunk * r);
    FA_CHECK_CUDA(cudaMemcpyAsync(dtop.p, top, sizeof(float) * (size_t)ntop * d, cudaMemcpyHostToDevice, st));
    FA_CHECK_CUDA(cudaMemcpyAsync(dl.p, lists, sizeof(float) * (size_t)nlist * d, cudaMemcpyHostToDevice, st));
    FA_CHECK_CUDA(cudaMemcpyAsync(dsb.p, sub_beg, sizeof(int32_t) * ((size_t)ntop + 1),
                                  cudaMemcpyHostToDevice, st));
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t cnt = std::min(chunk, n - r0);
        const unsigned g = (unsigned)((cnt + TILE - 1) / TILE);
        rows_to_f32(rows, r0, cnt, d, dt, dx.as<float>(), ds.as<uint8_t>(), st);
        // the TP nearest top-level clusters of every row
        k_l2_topr<<<g, 256, 0, st>>>(dx.as<float>(), nullptr, cnt, d, dtop.as<float>(), ntop, nullptr,
                                     nullptr, TP, dsup.as<int32_t>(), nullptr);
        FA_CHECK_CUDA(cudaGetLastError());
        for (int32_t j = 0; j < TP; ++j) {
            // rows grouped by their j-th cluster, so a CTA's rows share their lists
            launch_query_order(dsup.as<int32_t>() + j, cnt, TP, ntop, dcnt.as<uint32_t>(),
                               dord.as<int32_t>(), st);
            k_seg_ranges<<<1024, 256, 0, st>>>(dord.as<int32_t>(), dsup.as<int32_t>() + j, TP, cnt,
                                               dsb.as<int32_t>(), ntop, dcb.as<int32_t>(), dce.as<int32_t>());
            int32_t *ti = j == 0 ? di.as<int32_t>() : dj.as<int32_t>();
            float *td = j == 0 ? dd2.as<float>() : ddj.as<float>();
            k_l2_topr<<<g, 256, 0, st>>>(dx.as<float>(), dord.as<int32_t>(), cnt, d, dl.as<float>(), nlist,
                                         dcb.as<int32_t>(), dce.as<int32_t>(), r, ti, td);
            FA_CHECK_CUDA(cudaGetLastError());
            if (j > 0) {
                k_merge_topr<<<1024, 256, 0, st>>>(di.as<int32_t>(), dd2.as<float>(), dj.as<int32_t>(),
                                                   ddj.as<float>(), cnt, r);
                FA_CHECK_CUDA(cudaGetLastError());
            }
        }
        FA_CHECK_CUDA(cudaMemcpyAsync(out_ids + r0 * r, di.p, sizeof(int32_t) * cnt * r,
                                      cudaMemcpyDeviceToHost, st));
        if (out_d2)
            FA_CHECK_CUDA(cudaMemcpyAsync(out_d2 + r0 * r, dd2.p, sizeof(float) * cnt * r,
                                          cudaMemcpyDeviceToHost, st));
        if (out_top)
            FA_CHECK_CUDA(cudaMemcpy2DAsync(out_top + r0, sizeof(int32_t), dsup.p, sizeof(int32_t) * TP,
                                            sizeof(int32_t), cnt, cudaMemcpyDeviceToHost, st));
        FA_CHECK_CUDA(cudaStreamSynchronize(st));
    }
    cudaStreamDestroy(st);
}

void gpu_encode(const void *rows, int64_t n, int32_t d, fa_dtype dt, const float *codebooks,
                int32_t M, uint8_t *out_codes) {
    FA_REQUIRE(d / M <= 16, FA_ERR_ARG, "d/M above 16");
    cudaStream_t st;
    FA_CHECK_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    const int64_t chunk = 1 << 18;
    DevBuf dcb(sizeof(float) * (size_t)d * 256), dx(sizeof(float) * chunk * d), ds((size_t)chunk * d),
        dcode((size_t)chunk * M);
    FA_CHECK_CUDA(cudaMemcpyAsync(dcb.p, codebooks, sizeof(float) * (size_t)d * 256,
                                  cudaMemcpyHostToDevice, st));
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t cnt = std::min(chunk, n - r0);
        rows_to_f32(rows, r0, cnt, d, dt, dx.as<float>(), ds.as<uint8_t>(), st);
        const int64_t tot = cnt * M;
        k_encode<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(dx.as<float>(), cnt, d,
                                                               dcb.as<float>(), M, dcode.as<uint8_t>());
        FA_CHECK_CUDA(cudaGetLastError());
        FA_CHECK_CUDA(cudaMemcpyAsync(out_codes + r0 * M, dcode.p, (size_t)cnt * M,
                                      cudaMemcpyDeviceToHost, st));
        FA_CHECK_CUDA(cudaStreamSynchronize(st));
    }
    cudaStreamDestroy(st);
}

int num_sms(int device) {
    static int cached[64] = {0};
    if (device < 0 || device >= 64) device = 0;
    if (!cached[device]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0)
            v = 148;
        cached[device] = v;
    }
    return cached[device];
}

int cur_num_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    return num_sms(dev);
}

// ---------------------------------------------------------------------------
// Coarse probe that allocates nothing.
//
// Some callers cannot call cudaMalloc: processes whose device memory is owned
// in full by another allocator (a framework's caching pool, a fixed memory
// budget carved up at start-up), and latency-bound callers that cannot afford
// the device-wide synchronisation and unbounded time an allocation may take in
// the middle of their work. For them the distance block of the coarse probe
// lives in the file-scope array below, which every GPU that loads this library
// keeps for the life of the process (16 MiB). The caller still passes the
// queries, the centroids and the output.
//
// The array is shared by every call and keeps the last call's contents; each
// call overwrites every element it later reads, so nothing has to start at
// zero. Calls that overlap on the GPU (two streams, or two host threads) race
// on the array and may return wrong probe lists: serialise them.
// ---------------------------------------------------------------------------
constexpr int64_t NOALLOC_SCRATCH_FLOATS = 4ll << 20;
static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_SCRATCH_FLOATS];

// Device address of the array on the current device, looked up once per device
// with that device current (in host code the symbol is only a stand-in).
static float *noalloc_scratch() {
    static std::mutex mu;
    static float *addr[64] = {nullptr};
    int dev = 0;
    FA_CHECK_CUDA(cudaGetDevice(&dev));
    FA_REQUIRE(dev >= 0 && dev < 64, FA_ERR_NODEV, "device ordinal above 63");
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        float *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            throw Error{FA_ERR_CUDA, std::string("cudaGetSymbolAddress of the no-alloc scratch: ") +
                                         cudaGetErrorString(e)};
        addr[dev] = p;
    }
    return addr[dev];
}

}  // namespace fa

extern "C" fa_status fa_coarse_probe_noalloc(const float *queries, int64_t nq, int32_t d,
                                             const float *centroids, int32_t nlist, int32_t nprobe,
                                             int32_t *probes, void *stream) {
    using namespace fa;
    try {
        FA_REQUIRE(nq >= 0 && d >= 1 && nlist >= 1, FA_ERR_ARG, "bad shape");
        FA_REQUIRE(nprobe >= 1 && nprobe <= 512 && nprobe <= nlist, FA_ERR_ARG,
                   "nprobe must be in 1..min(nlist, 512)");
        FA_REQUIRE((int64_t)nlist <= NOALLOC_SCRATCH_FLOATS, FA_ERR_ARG,
                   "nlist above the no-alloc scratch capacity of 4194304 distances");
        if (nq == 0) return FA_OK;
        FA_REQUIRE(queries && centroids && probes, FA_ERR_ARG, "null buffer");
        float *scratch = noalloc_scratch();
        const int64_t rows = NOALLOC_SCRATCH_FLOATS / nlist;  // query rows per block
        l2_topn(queries, nq, d, centroids, nlist, nprobe, scratch, rows, probes, nprobe, nullptr,
                (cudaStream_t)stream);
        return FA_OK;
    } catch (const Error &e) {
        set_error("%s", e.msg.c_str());
        return e.st;
    } catch (...) {
        set_error("unexpected internal error");
        return FA_ERR_CUDA;
    }
}
