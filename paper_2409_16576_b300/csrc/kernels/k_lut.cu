// Step 1 of the filtering path when the lookup table is materialised in HBM
// (the precision form): LUT[m][c] = dist(q_m, C_m[c]) for every subspace m and
// centroid c, stored as FP32, FP16 or FP8 (e4m3).
//
// Quantised tables keep, per query, one scale s and per subspace an offset
// o_m = min_c LUT[m][c]:  LUT[m][c] ~= s * stored[m][c] + o_m,
// stored = round(( LUT[m][c] - o_m ) / s) with s = max residual / format max.
// The ADC scan dequantises into its FP32 shared-memory table, so sums stay
// FP32; each entry is off by at most half a unit in the last place of the
// stored value times s.
//
// lut_scale row layout per query: [0] = s, [1] = sum_m o_m, [2 + m] = o_m.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "../fa_internal.h"

namespace fa {

constexpr float F16_MAX = 65504.f;
constexpr float FP8_MAX = 448.f;

__device__ __forceinline__ float block_reduce_max(float v, float *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) red[0] = v;
    }
    __syncthreads();
    v = red[0];
    __syncthreads();
    return v;
}

// Stores a FP32 table held in shared memory (t[m*256 + c]) in the requested
// precision, with per-subspace offsets and a per-query scale.
__device__ void store_lut(const float *t, int M, int prec, void *lut, float *scale, int64_t qi,
                          float *red, float *offs) {
    const int64_t base = qi * (int64_t)M * 256;
    float *sc = scale + qi * (2 + M);
    if (prec == FA_LUT_F32) {
        for (int i = threadIdx.x; i < M * 256; i += blockDim.x)
            reinterpret_cast<float *>(lut)[base + i] = t[i];
        if (threadIdx.x == 0) {
            sc[0] = 1.f;
            sc[1] = 0.f;
        }
        for (int m = threadIdx.x; m < M; m += blockDim.x) sc[2 + m] = 0.f;
        return;
    }
    // per-subspace minimum: one warp per subspace
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int m = warp; m < M; m += nw) {
        float v = INFINITY;
        for (int c = lane; c < 256; c += 32) v = fminf(v, t[m * 256 + c]);
        for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) offs[m] = v;
    }
    __syncthreads();
    float mx = 0.f;
    for (int i = threadIdx.x; i < M * 256; i += blockDim.x) mx = fmaxf(mx, t[i] - offs[i >> 8]);
    mx = block_reduce_max(mx, red);
    const float fmax = prec == FA_LUT_F16 ? F16_MAX : FP8_MAX;
    float s = mx / fmax;
    if (!(s > 0.f)) s = 1.f;
    const float inv = 1.f / s;
    for (int i = threadIdx.x; i < M * 256; i += blockDim.x) {
        const float r = fminf((t[i] - offs[i >> 8]) * inv, fmax);
        if (prec == FA_LUT_F16) {
            reinterpret_cast<__half *>(lut)[base + i] = __float2half_rn(r);
        } else {
            const __nv_fp8_e4m3 v(r);
            reinterpret_cast<uint8_t *>(lut)[base + i] = v.__x;
        }
    }
    if (threadIdx.x == 0) {
        float so = 0.f;
        for (int m = 0; m < M; ++m) so += offs[m];
        sc[0] = s;
        sc[1] = so;
    }
    for (int m = threadIdx.x; m < M; m += blockDim.x) sc[2 + m] = offs[m];
}

// FP32 direct differences, one CTA per query.
__global__ void __launch_bounds__(256) k_lut_simt(const float *__restrict__ q, int64_t nq, int32_t d,
                                                  const float *__restrict__ cb, int32_t M, int prec,
                                                  void *lut, float *scale) {
    extern __shared__ float sm[];
    float *t = sm;                 // [M][256]
    float *qv = t + M * 256;       // [d]
    float *offs = qv + d;          // [M]
    __shared__ float red[32];
    const int dsub = d / M;
    for (int64_t qi = blockIdx.x; qi < nq; qi += gridDim.x) {
        for (int j = threadIdx.x; j < d; j += blockDim.x) qv[j] = q[qi * d + j];
        __syncthreads();
        for (int i = threadIdx.x; i < M * 256; i += blockDim.x) {
            const int m = i >> 8, c = i & 255;
            const float *w = cb + ((int64_t)m * 256 + c) * dsub;
            float s = 0.f;
            for (int j = 0; j < dsub; ++j) {
                const float df = qv[m * dsub + j] - w[j];
                s = fmaf(df, df, s);
            }
            t[i] = s;
        }
        __syncthreads();
        store_lut(t, M, prec, lut, scale, qi, red, offs);
        __syncthreads();
    }
}

void launch_lut_tc(const DeviceIndex &ix, const float *q, int64_t nq, int prec, void *lut,
                   float *lut_scale, cudaStream_t st);

void launch_lut_global(const DeviceIndex &ix, const float *q, int64_t nq, int prec, int gemm,
                       void *lut, float *lut_scale, cudaStream_t st) {
    if (nq == 0) return;
    if (gemm == FA_GEMM_BF16_TC) {
        launch_lut_tc(ix, q, nq, prec, lut, lut_scale, st);
        return;
    }
    const int smem = (ix.M * 256 + ix.d + ix.M) * 4;
    FA_CHECK_CUDA(cudaFuncSetAttribute(k_lut_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int grid = (int)std::min<int64_t>(nq, (int64_t)num_sms(0) * 4);
    k_lut_simt<<<grid, 256, smem, st>>>(q, nq, ix.d, ix.codebooks, ix.M, prec, lut, lut_scale);
    FA_CHECK_CUDA(cudaGetLastError());
}

}  // namespace fa
