// Step 1 of the filtering path when the lookup table is materialised in HBM
// (the precision form): LUT[m][c] = dist(q_m, C_m[c]) for every subspace m and
// centroid c, stored as FP32, FP16 or FP8 (e4m3).
//
// Quantised tables keep, per query and subspace m, a scale s_m and an offset
// o_m = min_c LUT[m][c]:  LUT[m][c] ~= s_m * stored[m][c] + o_m, with
// stored = round((LUT[m][c] - o_m) / s_m) and s_m = (max - min) / format max.
// The ADC scan dequantises into its FP32 shared-memory table, so sums stay
// FP32; each entry is off by at most half a unit in the last place of the
// stored value times s_m.
//
// lut_scale row layout per query: [2m] = s_m, [2m + 1] = o_m. With a uniform
// scale (the batched form, which adds stored entries directly) every s_m is
// the same per-query s_q: here the largest subspace scale, in the tensor-core
// kernel a bound that needs no pass over the other subspaces.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "../fa_internal.h"

namespace fa {

constexpr float F16_MAX = 65504.f;
constexpr float FP8_MAX = 448.f;

// Stores a FP32 table held in shared memory (t[m*256 + c]) in the requested
// precision with a per-subspace scale and offset.
__device__ void store_lut(const float *t, int M, int Mr, int prec, void *lut, float *scale, int64_t qi,
                          float *offs, float *scl, int uniform) {
    const int64_t base = qi * (int64_t)M * 256;
    float *sc = scale + qi * 2 * M;
    if (prec == FA_LUT_F32) {
        for (int i = threadIdx.x; i < M * 256; i += blockDim.x)
            reinterpret_cast<float *>(lut)[base + i] = t[i];
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            sc[2 * m] = 1.f;
            sc[2 * m + 1] = 0.f;
        }
        return;
    }
    // per-subspace minimum and maximum: one warp per subspace
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float fmax = prec == FA_LUT_F16 ? F16_MAX : FP8_MAX;
    for (int m = warp; m < M; m += nw) {
        float lo = INFINITY, hi = -INFINITY;
        for (int c = lane; c < 256; c += 32) {
            lo = fminf(lo, t[m * 256 + c]);
            hi = fmaxf(hi, t[m * 256 + c]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        float s = (hi - lo) / fmax;
        if (!(s > 0.f)) s = 1.f;
        if (m >= Mr) s = lo = 0.f;  // padding subspace: every entry 0
        if (lane == 0) {
            offs[m] = lo;
            scl[m] = s;
        }
    }
    __syncthreads();
    // uniform: the largest subspace scale serves every subspace
    float su = 0.f;
    if (uniform)
        for (int m = 0; m < M; ++m) su = fmaxf(su, scl[m]);
    __syncthreads();
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        if (uniform) scl[m] = su;
        sc[2 * m] = scl[m];
        sc[2 * m + 1] = offs[m];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < M * 256; i += blockDim.x) {
        const int m = i >> 8;
        const float r = scl[m] > 0.f ? fminf((t[i] - offs[m]) / scl[m], fmax) : 0.f;
        if (prec == FA_LUT_F16) {
            reinterpret_cast<__half *>(lut)[base + i] = __float2half_rn(r);
        } else {
            const __nv_fp8_e4m3 v(r);
            reinterpret_cast<uint8_t *>(lut)[base + i] = v.__x;
        }
    }
}

// FP32 direct differences, one CTA per query.
__global__ void __launch_bounds__(256) k_lut_simt(const float *__restrict__ q, int64_t nq, int32_t d,
                                                  const float *__restrict__ cb, int32_t M, int32_t Mr,
                                                  int prec, void *lut, float *scale, int uniform, int ip) {
    extern __shared__ float sm[];
    float *t = sm;                 // [M][256]
    float *qv = t + M * 256;       // [d]
    float *offs = qv + d;          // [M]
    float *scl = offs + M;         // [M]
    const int dsub = d / Mr;
    for (int64_t qi = blockIdx.x; qi < nq; qi += gridDim.x) {
        for (int j = threadIdx.x; j < d; j += blockDim.x) qv[j] = q[qi * d + j];
        __syncthreads();
        for (int i = threadIdx.x; i < M * 256; i += blockDim.x) {
            const int m = i >> 8, c = i & 255;
            float s = 0.f;
            if (m < Mr) {  // padding subspaces stay 0
                const float *w = cb + ((int64_t)m * 256 + c) * dsub;
                for (int j = 0; j < dsub; ++j) {
                    if (ip) {  // inner product: -<q_m, C_m[c]>
                        s = fmaf(-qv[m * dsub + j], w[j], s);
                    } else {
                        const float df = qv[m * dsub + j] - w[j];
                        s = fmaf(df, df, s);
                    }
                }
            }
            t[i] = s;
        }
        __syncthreads();
        store_lut(t, M, Mr, prec, lut, scale, qi, offs, scl, uniform);
        __syncthreads();
    }
}

void launch_lut_tc(const DeviceIndex &ix, const float *q, int64_t nq, int prec, void *lut,
                   float *lut_scale, uint32_t *err, cudaStream_t st, int uniform);

void launch_lut_global(const DeviceIndex &ix, const float *q, int64_t nq, int prec, int gemm,
                       void *lut, float *lut_scale, uint32_t *err, cudaStream_t st, int uniform) {
    if (nq == 0) return;
    if (gemm == FA_GEMM_BF16_TC) {
        launch_lut_tc(ix, q, nq, prec, lut, lut_scale, err, st, uniform);
        return;
    }
    const int smem = (ix.Mp * 256 + ix.d + 2 * ix.Mp) * 4;
    FA_CHECK_CUDA(cudaFuncSetAttribute(k_lut_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int grid = (int)std::min<int64_t>(nq, (int64_t)cur_num_sms() * 4);
    k_lut_simt<<<grid, 256, smem, st>>>(q, nq, ix.d, ix.codebooks, ix.Mp, ix.M, prec, lut, lut_scale,
                                        uniform, ix.metric == FA_METRIC_IP ? 1 : 0);
    FA_CHECK_CUDA(cudaGetLastError());
}

}  // namespace fa
