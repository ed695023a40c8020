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
// The epilogue reads each query row's 256 entries back from tensor memory
// twice: once for the subspace's minimum and maximum, once to store the
// entries as FP32, or as FP16 / FP8 with that subspace's scale and offset
// (stored = (LUT - min) / s, s = (max - min) / format max).
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <vector>

#include "../fa_internal.h"
#include "tc_util.cuh"

namespace fa {

constexpr int LQ = 128;   // queries per tile
constexpr int LN = 256;   // centroids per subspace
constexpr int LSUB = 8;   // subspaces per CTA
constexpr uint32_t LUT_WAIT_LIMIT = 1u << 22;

struct LutTcArgs {
    const float *q;
    int64_t nq;
    int32_t d, Kp, M, dsub;
    const __nv_bfloat16 *btiles;  // [M][hi, lo][LN x 16] core-matrix layout
    const float *cbnorm;          // [M][256] |C_m[c]|^2
    int32_t prec;
    void *lut;                    // [nq][M][256]
    float *scale;                 // [nq][2M]: (s_m, o_m)
    uint32_t *err;
};

__global__ void __launch_bounds__(LQ, 1) k_lut_tc(const LutTcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int Kp = a.Kp;
    __nv_bfloat16 *Ahi = reinterpret_cast<__nv_bfloat16 *>(sm);
    __nv_bfloat16 *Alo = Ahi + LQ * Kp;
    __nv_bfloat16 *Bt = Alo + LQ * Kp;  // hi then lo, 2 * LN * 16
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * LQ;
    const int64_t row = r0 + tid;
    const bool row_ok = row < a.nq;

    for (int e = tid; e < LQ * Kp; e += LQ) {
        const int r = e / Kp, k = e - r * Kp;
        const float x = (r0 + r < a.nq && k < a.d) ? a.q[(r0 + r) * a.d + k] : 0.f;
        __nv_bfloat16 h, l;
        tc::split_bf16(x, h, l);
        const uint32_t o = tc::core_offset(r, k, Kp) >> 1;
        Ahi[o] = h;
        Alo[o] = l;
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, LN);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = tmem_base;
    const uint32_t lane_addr = tbase + ((uint32_t)(warp * 32) << 16);
    const uint32_t idesc = tc::idesc_bf16_f32(LQ, LN);
    const uint32_t sbo_a = (uint32_t)(Kp / 8) * 128u, sbo_b = 256u;
    uint32_t parity = 0;
    bool failed = false;
    const int m0 = blockIdx.y * LSUB, m1 = min(a.M, m0 + LSUB);
    const float fmax = a.prec == FA_LUT_F16 ? 65504.f : 448.f;

    for (int m = m0; m < m1; ++m) {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.btiles + (size_t)m * 2 * LN * 16);
        uint4 *dst = reinterpret_cast<uint4 *>(Bt);
        for (int i = tid; i < 2 * LN * 16 * 2 / 16; i += LQ) dst[i] = __ldg(src + i);
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
            const uint32_t off = 256u * (uint32_t)((m * a.dsub) / 16);
            const uint64_t dah = tc::smem_desc(tc::smem_u32(Ahi) + off, 128, sbo_a);
            const uint64_t dal = tc::smem_desc(tc::smem_u32(Alo) + off, 128, sbo_a);
            const uint32_t bh = tc::smem_u32(Bt), bl = bh + LN * 16 * 2;
            const uint64_t dbh = tc::smem_desc(bh, 128, sbo_b);
            const uint64_t dbl = tc::smem_desc(bl, 128, sbo_b);
            tc::mma_bf16(tbase, dah, dbh, idesc, 0u);
            tc::mma_bf16(tbase, dah, dbl, idesc, 1u);
            tc::mma_bf16(tbase, dal, dbh, idesc, 1u);
            tc::mma_commit(&mbar);
        }
        const bool ok = tc::mbar_wait(&mbar, parity, LUT_WAIT_LIMIT);
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
        if (a.prec != FA_LUT_F32) {
#pragma unroll 1
            for (int c0 = 0; c0 < LN; c0 += 32) {
                float v[32];
                tc::tmem_ld32(lane_addr + c0, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float e = qn - 2.f * v[i] + __ldg(cn + c0 + i);
                    lo = fminf(lo, e);
                    hi = fmaxf(hi, e);
                }
            }
        }
        float s = (hi - lo) / fmax;
        if (!(s > 0.f)) s = 1.f;
        const float inv = 1.f / s;
        const int64_t base = (row * a.M + m) * 256;
#pragma unroll 1
        for (int c0 = 0; c0 < LN; c0 += 32) {
            float v[32];
            tc::tmem_ld32(lane_addr + c0, v);
            if (!row_ok) continue;
            if (a.prec == FA_LUT_F32) {
                float4 *o = reinterpret_cast<float4 *>(reinterpret_cast<float *>(a.lut) + base + c0);
#pragma unroll
                for (int i = 0; i < 32; i += 4)
                    o[i / 4] = make_float4(qn - 2.f * v[i] + __ldg(cn + c0 + i),
                                           qn - 2.f * v[i + 1] + __ldg(cn + c0 + i + 1),
                                           qn - 2.f * v[i + 2] + __ldg(cn + c0 + i + 2),
                                           qn - 2.f * v[i + 3] + __ldg(cn + c0 + i + 3));
            } else if (a.prec == FA_LUT_F16) {
                uint32_t w[16];
#pragma unroll
                for (int i = 0; i < 32; i += 2) {
                    const float e0 = fminf((qn - 2.f * v[i] + __ldg(cn + c0 + i) - lo) * inv, fmax);
                    const float e1 =
                        fminf((qn - 2.f * v[i + 1] + __ldg(cn + c0 + i + 1) - lo) * inv, fmax);
                    const __half2 h = __floats2half2_rn(e0, e1);
                    w[i / 2] = *reinterpret_cast<const uint32_t *>(&h);
                }
                uint4 *o = reinterpret_cast<uint4 *>(reinterpret_cast<__half *>(a.lut) + base + c0);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    o[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
            } else {
                uint32_t w[8];
#pragma unroll
                for (int i = 0; i < 32; i += 4) {
                    uint32_t pk = 0;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float e =
                            fminf((qn - 2.f * v[i + j] + __ldg(cn + c0 + i + j) - lo) * inv, fmax);
                        const __nv_fp8_e4m3 f(e);
                        pk |= (uint32_t)f.__x << (8 * j);
                    }
                    w[i / 4] = pk;
                }
                uint4 *o = reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(a.lut) + base + c0);
                o[0] = make_uint4(w[0], w[1], w[2], w[3]);
                o[1] = make_uint4(w[4], w[5], w[6], w[7]);
            }
        }
        if (row_ok) {
            a.scale[row * 2 * a.M + 2 * m] = a.prec == FA_LUT_F32 ? 1.f : s;
            a.scale[row * 2 * a.M + 2 * m + 1] = a.prec == FA_LUT_F32 ? 0.f : lo;
        }
        tc::fence_before();
        __syncthreads();
    }
    if (failed) {
        if (tid == 0 && a.err) atomicOr(a.err, DEV_ERR_TIMEOUT);
        tc::mbar_wait(&mbar, parity, LUT_WAIT_LIMIT);
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
                   float *lut_scale, uint32_t *err, cudaStream_t st) {
    FA_REQUIRE(ix.codebooks_bf16 != nullptr, FA_ERR_ARG,
               "the tensor-core LUT needs d <= 128 and d / M dividing 16");
    LutTcArgs a{};
    a.q = q;
    a.nq = nq;
    a.d = ix.d;
    a.Kp = ix.tc_kp;
    a.M = ix.M;
    a.dsub = ix.dsub;
    a.btiles = reinterpret_cast<const __nv_bfloat16 *>(ix.codebooks_bf16);
    a.cbnorm = ix.cbnorm;
    a.prec = prec;
    a.lut = lut;
    a.scale = lut_scale;
    a.err = err;
    // at least 80 KB so that at most two CTAs (2 x 256 TMEM columns) share an SM
    const int smem = std::max((2 * LQ * a.Kp + 2 * LN * 16) * 2, 80 * 1024);
    FA_CHECK_CUDA(cudaFuncSetAttribute(k_lut_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const dim3 grid((unsigned)((nq + LQ - 1) / LQ), (unsigned)((ix.M + LSUB - 1) / LSUB));
    k_lut_tc<<<grid, LQ, smem, st>>>(a);
    FA_CHECK_CUDA(cudaGetLastError());
}

}  // namespace fa
