// LUT build (step 1) on the tensor cores:
//   LUT[q][m][c] = |q_m|^2 - 2 q_m . C_m[c] + |C_m[c]|^2
// The dot products of all M subspaces form a block-diagonal GEMM of the
// queries against the M x 256 sub-codebooks. Subspace m covers d/M <= 16
// coordinates, which sit inside one K = 16 step of the query tile; its B
// operand is a 256 x 16 tile holding C_m's coordinates in their columns and
// zeros elsewhere (prepared at index upload). One MMA group per subspace
// (M = 128 queries, N = 256 centroids, K = 16) accumulates in tensor memory;
// queries and codebooks are split into bf16 hi + lo pairs and take three MMAs
// (hi.hi + hi.lo + lo.hi) so the dot products come out near FP32.
//
// A CTA takes 128 queries and LSUB subspaces. It converts only the K-blocks
// those subspaces use, and double-buffers the subspaces' B tiles with bulk
// copies, so that a tile arrives while the previous subspace's epilogue runs.
// The epilogue reads each query row's 256 entries back from tensor memory
// twice: once for the subspace's minimum and maximum, once to store the
// entries as FP32, or as FP16 / FP8 with that subspace's scale and offset
// (stored = (LUT - min) / s, s = (max - min) / format max). FP16 / FP8 rows are
// staged in shared memory and written back one whole row per warp store.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <vector>

#include "../fa_internal.h"
#include "tc_util.cuh"

namespace fa {

constexpr int LQ = 128;   // queries per tile
constexpr int LN = 256;   // centroids per subspace
constexpr int LSUB = 4;   // subspaces per CTA
constexpr int STAGE_PAD = 16;  // bytes after each staged row: rows start in different banks
constexpr uint32_t LUT_WAIT_LIMIT = 1u << 22;

struct LutTcArgs {
    const float *q;
    int64_t nq;
    int32_t d, Kp, M, dsub;
    int32_t Mp;                   // table rows per query (M rounded up to the scan width)
    const __nv_bfloat16 *btiles;  // [M][hi, lo][LN x 16] core-matrix layout
    const float *cbnorm;          // [M][256] |C_m[c]|^2
    int32_t prec;
    void *lut;                    // [nq][M][256]
    float *scale;                 // [nq][2M]: (s_m, o_m)
    uint32_t *err;
    int32_t uniform;              // one scale per query: s_q = 2 (|q|^2 + max |C_m[c]|^2) / format max
    float cmax2;                  // max over m, c of |C_m[c]|^2
    int32_t ip;                   // entries -q_m.C_m[c] (inner product) instead of the squared L2
};

__host__ __device__ inline int lut_elem(int prec) {
    return prec == FA_LUT_F16 ? 2 : (prec == FA_LUT_FP8 ? 1 : 4);
}

__global__ void __launch_bounds__(LQ, 1) k_lut_tc(const LutTcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar, full[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * LSUB, m1 = min(a.M, m0 + LSUB);
    // only the 16-wide K-blocks this CTA's subspaces use
    const int kb0 = (m0 * a.dsub) / 16, kb1 = (m1 * a.dsub + 15) / 16;
    const int Ka = (kb1 - kb0) * 16;
    const uint32_t btile = 2u * LN * 16 * 2;  // hi + lo of one subspace
    const bool staged = a.prec != FA_LUT_F32;
    const int elem = lut_elem(a.prec), srow = LN * elem + STAGE_PAD;
    __nv_bfloat16 *Ahi = reinterpret_cast<__nv_bfloat16 *>(sm);
    __nv_bfloat16 *Alo = Ahi + LQ * Ka;
    unsigned char *Bb = sm + (size_t)2 * LQ * Ka * 2;  // two subspace tiles
    unsigned char *stage = Bb + 2 * btile;             // [LQ][srow] quantised rows
    const int64_t r0 = (int64_t)blockIdx.x * LQ;
    const int64_t row = r0 + tid;
    const bool row_ok = row < a.nq;

    for (int e = tid; e < LQ * Ka; e += LQ) {
        const int r = e / Ka, k = e - r * Ka, gk = kb0 * 16 + k;
        const float x = (r0 + r < a.nq && gk < a.d) ? a.q[(r0 + r) * a.d + gk] : 0.f;
        __nv_bfloat16 h, l;
        tc::split_bf16(x, h, l);
        const uint32_t o = tc::core_offset(r, k, Ka) >> 1;
        Ahi[o] = h;
        Alo[o] = l;
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, LN);
    if (tid == 0) {
        tc::mbar_init(&mbar, 1);
        tc::mbar_init(&full[0], 1);
        tc::mbar_init(&full[1], 1);
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = tmem_base;
    const uint32_t lane_addr = tbase + ((uint32_t)(warp * 32) << 16);
    const uint32_t idesc = tc::idesc_bf16_f32(LQ, LN);
    const uint32_t sbo_a = (uint32_t)(Ka / 8) * 128u, sbo_b = 256u;
    uint32_t parity = 0;
    bool failed = false;
    int loaded = -1;  // last subspace whose tile copy thread 0 issued
    const float fmax = a.prec == FA_LUT_F16 ? 65504.f : 448.f;
    // uniform scale: every entry |q_m - C_m[c]|^2 is at most 2 (|q_m|^2 + |C_m[c]|^2)
    // <= 2 (|q|^2 + cmax2), so the stored residuals stay within the format
    float su = 1.f;
    if (a.uniform && row_ok) {
        float qq = 0.f;
        for (int j = 0; j < a.d; ++j) {
            const float x = a.q[row * a.d + j];
            qq = fmaf(x, x, qq);
        }
        su = 2.f * (qq + a.cmax2) / fmax;
        if (!(su > 0.f)) su = 1.f;
    }
    if (tid == 0 && m0 < m1) {
        tc::mbar_expect_tx(&full[0], btile);
        tc::bulk_g2s(Bb, a.btiles + (size_t)m0 * 2 * LN * 16, btile, &full[0]);
        loaded = m0;
    }

    for (int m = m0; m < m1; ++m) {
        const int i = m - m0, b = i & 1;
        if (tid == 0) {
            bool ok0 = tc::mbar_wait(&full[b], (i >> 1) & 1, LUT_WAIT_LIMIT);
            if (ok0) {
                tc::fence_after();
                const uint32_t off = 256u * (uint32_t)((m * a.dsub) / 16 - kb0);
                const uint64_t dah = tc::smem_desc(tc::smem_u32(Ahi) + off, 128, sbo_a);
                const uint64_t dal = tc::smem_desc(tc::smem_u32(Alo) + off, 128, sbo_a);
                const uint32_t bh = tc::smem_u32(Bb + (size_t)b * btile), bl = bh + LN * 16 * 2;
                const uint64_t dbh = tc::smem_desc(bh, 128, sbo_b);
                const uint64_t dbl = tc::smem_desc(bl, 128, sbo_b);
                tc::mma_bf16(tbase, dah, dbh, idesc, 0u);
                tc::mma_bf16(tbase, dah, dbl, idesc, 1u);
                tc::mma_bf16(tbase, dal, dbh, idesc, 1u);
                tc::mma_commit(&mbar);
                // the other tile buffer was read by subspace m - 1, whose MMAs are done
                if (m + 1 < m1) {
                    tc::mbar_expect_tx(&full[b ^ 1], btile);
                    tc::bulk_g2s(Bb + (size_t)(b ^ 1) * btile, a.btiles + (size_t)(m + 1) * 2 * LN * 16,
                                 btile, &full[b ^ 1]);
                    loaded = m + 1;
                }
            }
            s_ok = ok0 ? 1 : 0;
        }
        __syncthreads();
        bool ok = s_ok != 0;
        ok = ok && tc::mbar_wait(&mbar, parity, LUT_WAIT_LIMIT);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        parity ^= 1u;
        tc::fence_after();

        float qn = 0.f;
        if (row_ok)
            for (int j = 0; j < a.dsub; ++j) {
                const float x = a.q[row * a.d + m * a.dsub + j];
                qn = fmaf(x, x, qn);
            }
        const float *cn = a.cbnorm + m * 256;
        float lo = INFINITY, hi = -INFINITY;
        if (staged) {
#pragma unroll 1
            for (int c0 = 0; c0 < LN; c0 += 32) {
                float v[32];
                tc::tmem_ld32(lane_addr + c0, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float e = a.ip ? -v[j] : qn - 2.f * v[j] + __ldg(cn + c0 + j);
                    lo = fminf(lo, e);
                    hi = fmaxf(hi, e);
                }
            }
        }
        float s = a.uniform ? su : (hi - lo) / fmax;
        if (!(s > 0.f)) s = 1.f;
        const float inv = 1.f / s;
        const int64_t base = (row * a.Mp + m) * 256;
        unsigned char *srw = stage + (size_t)tid * srow;
#pragma unroll 1
        for (int c0 = 0; c0 < LN; c0 += 32) {
            float v[32];
            tc::tmem_ld32(lane_addr + c0, v);
            if (a.prec == FA_LUT_F32) {
                if (!row_ok) continue;
                float4 *o = reinterpret_cast<float4 *>(reinterpret_cast<float *>(a.lut) + base + c0);
#pragma unroll
                for (int j = 0; j < 32; j += 4)
                    o[j / 4] = a.ip ? make_float4(-v[j], -v[j + 1], -v[j + 2], -v[j + 3])
                                    : make_float4(qn - 2.f * v[j] + __ldg(cn + c0 + j),
                                                  qn - 2.f * v[j + 1] + __ldg(cn + c0 + j + 1),
                                                  qn - 2.f * v[j + 2] + __ldg(cn + c0 + j + 2),
                                                  qn - 2.f * v[j + 3] + __ldg(cn + c0 + j + 3));
            } else if (a.prec == FA_LUT_F16) {
                uint32_t w[16];
#pragma unroll
                for (int j = 0; j < 32; j += 2) {
                    const float x0 = a.ip ? -v[j] : qn - 2.f * v[j] + __ldg(cn + c0 + j);
                    const float x1 = a.ip ? -v[j + 1] : qn - 2.f * v[j + 1] + __ldg(cn + c0 + j + 1);
                    const float e0 = fminf((x0 - lo) * inv, fmax);
                    const float e1 = fminf((x1 - lo) * inv, fmax);
                    const __half2 h = __floats2half2_rn(e0, e1);
                    w[j / 2] = *reinterpret_cast<const uint32_t *>(&h);
                }
                uint4 *o = reinterpret_cast<uint4 *>(srw + c0 * 2);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    o[j] = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
            } else {
                uint32_t w[8];
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    uint32_t pk = 0;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const float xe = a.ip ? -v[j + t] : qn - 2.f * v[j + t] + __ldg(cn + c0 + j + t);
                        const float e = fminf((xe - lo) * inv, fmax);
                        const __nv_fp8_e4m3 f(e);
                        pk |= (uint32_t)f.__x << (8 * t);
                    }
                    w[j / 4] = pk;
                }
                uint4 *o = reinterpret_cast<uint4 *>(srw + c0);
                o[0] = make_uint4(w[0], w[1], w[2], w[3]);
                o[1] = make_uint4(w[4], w[5], w[6], w[7]);
            }
        }
        if (row_ok) {
            a.scale[row * 2 * a.Mp + 2 * m] = staged ? s : 1.f;
            a.scale[row * 2 * a.Mp + 2 * m + 1] = staged ? lo : 0.f;
        }
        tc::fence_before();
        __syncthreads();  // the staged tile is complete and the accumulator free
        if (staged) {
            // one query row per warp store: a row of the subspace is LN * elem
            // contiguous bytes in HBM
            for (int r = warp; r < LQ; r += LQ / 32) {
                if (r0 + r >= a.nq) break;
                unsigned char *dst = reinterpret_cast<unsigned char *>(a.lut) + ((r0 + r) * a.Mp + m) * 256 * elem;
                const unsigned char *src = stage + (size_t)r * srow;
                if (elem == 2)
                    reinterpret_cast<uint4 *>(dst)[lane] = reinterpret_cast<const uint4 *>(src)[lane];
                else
                    reinterpret_cast<uint2 *>(dst)[lane] = reinterpret_cast<const uint2 *>(src)[lane];
            }
            __syncthreads();  // the stage takes the next subspace
        }
    }
    if (failed) {
        if (tid == 0) {
            if (a.err) atomicOr(a.err, DEV_ERR_TIMEOUT);
            // copies and MMAs in flight finish before shared and tensor memory go
            tc::mbar_wait(&mbar, parity, LUT_WAIT_LIMIT);
            if (loaded >= m0) {
                const int li = loaded - m0;
                tc::mbar_wait(&full[li & 1], (li >> 1) & 1, LUT_WAIT_LIMIT);
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_free(tbase, LN);
}

// Per-subspace B tiles: [M][hi, lo][256 x 16] with C_m[c][j] in column
// (m * dsub) % 16 + j, zeros elsewhere; and |C_m[c]|^2 in FP32.
void prepare_codebook_tiles(const float *cb, int32_t M, int32_t d, std::vector<uint16_t> &tiles,
                            std::vector<float> &norms) {
    const int dsub = d / M;
    tiles.assign((size_t)M * 2 * LN * 16, 0);
    norms.assign((size_t)M * 256, 0.f);
    for (int m = 0; m < M; ++m) {
        uint16_t *hi = tiles.data() + (size_t)m * 2 * LN * 16;
        uint16_t *lo = hi + LN * 16;
        const int j0 = (m * dsub) % 16;
        for (int c = 0; c < 256; ++c) {
            double nrm = 0;
            for (int j = 0; j < dsub; ++j) {
                const float x = cb[((size_t)m * 256 + c) * dsub + j];
                const uint16_t h = tc::host_bf16_bits(x);
                const uint32_t o = tc::core_offset(c, j0 + j, 16) >> 1;
                hi[o] = h;
                lo[o] = tc::host_bf16_bits(x - tc::host_bf16_float(h));
                nrm += (double)x * x;
            }
            norms[(size_t)m * 256 + c] = (float)nrm;
        }
    }
}

void launch_lut_tc(const DeviceIndex &ix, const float *q, int64_t nq, int prec, void *lut,
                   float *lut_scale, uint32_t *err, cudaStream_t st, int uniform) {
    FA_REQUIRE(ix.codebooks_bf16 != nullptr, FA_ERR_ARG,
               "the tensor-core LUT needs d <= 128 and d / M dividing 16");
    LutTcArgs a{};
    a.q = q;
    a.nq = nq;
    a.d = ix.d;
    a.Kp = ix.tc_kp;
    a.M = ix.M;
    a.Mp = ix.Mp;
    a.dsub = ix.dsub;
    a.btiles = reinterpret_cast<const __nv_bfloat16 *>(ix.codebooks_bf16);
    a.cbnorm = ix.cbnorm;
    a.prec = prec;
    a.lut = lut;
    a.scale = lut_scale;
    a.err = err;
    a.uniform = uniform;
    a.cmax2 = ix.cb_max_norm2;
    a.ip = ix.metric == FA_METRIC_IP ? 1 : 0;
    // widest K-range of one CTA's subspaces (16-wide blocks), two tile buffers,
    // the staged rows; at least 80 KB so that at most two CTAs (2 x 256 TMEM
    // columns) share an SM
    int ka_max = 16;
    for (int m0 = 0; m0 < ix.M; m0 += LSUB) {
        const int m1 = std::min(ix.M, m0 + LSUB);
        ka_max = std::max(ka_max, ((m1 * ix.dsub + 15) / 16 - (m0 * ix.dsub) / 16) * 16);
    }
    const int stage = prec == FA_LUT_F32 ? 0 : LQ * (LN * lut_elem(prec) + STAGE_PAD);
    const int smem = std::max(2 * LQ * ka_max * 2 + 2 * 2 * LN * 16 * 2 + stage, 80 * 1024);
    FA_CHECK_CUDA(cudaFuncSetAttribute(k_lut_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const dim3 grid((unsigned)((nq + LQ - 1) / LQ), (unsigned)((ix.M + LSUB - 1) / LSUB));
    k_lut_tc<<<grid, LQ, smem, st>>>(a);
    FA_CHECK_CUDA(cudaGetLastError());
    if (ix.Mp > ix.M) {  // padding subspaces: zero entries, scale and offset 0
        const size_t row = (size_t)256 * lut_elem(prec);
        FA_CHECK_CUDA(cudaMemset2DAsync(static_cast<char *>(lut) + (size_t)ix.M * row, (size_t)ix.Mp * row,
                                        0, (size_t)(ix.Mp - ix.M) * row, (size_t)nq, st));
        FA_CHECK_CUDA(cudaMemset2DAsync(lut_scale + 2 * ix.M, sizeof(float) * 2 * ix.Mp, 0,
                                        sizeof(float) * 2 * (ix.Mp - ix.M), (size_t)nq, st));
    }
}

}  // namespace fa
