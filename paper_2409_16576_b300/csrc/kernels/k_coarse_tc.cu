// Coarse probe (step 2) distances on the tensor cores:
//   d2(q, c_l) = |q|^2 - 2 q.c_l + |c_l|^2
// for a tile of 128 queries x 256 centroids per MMA (M = 128, N = 256,
// K = 16 per instruction), accumulated in FP32 in tensor memory.
//
// Queries and centroids are both split into a bf16 pair hi + lo (x ~= hi +
// lo to ~16 significant bits) and the dot product takes three MMAs per K-step
// (hi.hi + hi.lo + lo.hi), so the product is close to FP32 accuracy while the
// contraction runs at bf16 tensor rate. The distances go to the per-call
// distance block and k_select picks the top-nprobe lists, as in the FP32 form.
//
// One CTA = 4 warps = 128 threads (one TMEM lane per thread). Thread 0 issues
// the MMAs and commits them to an mbarrier; every thread waits on it (with a
// bound) and reads its row's 256 accumulators back with tcgen05.ld.
#include <algorithm>
#include <vector>

#include "../fa_internal.h"
#include "tc_util.cuh"

namespace fa {

constexpr int TCQ = 128;                 // queries per tile (MMA M)
constexpr int TCN = 256;                 // centroids per tile (MMA N)
constexpr uint32_t WAIT_LIMIT = 1u << 22;

struct CoarseTcArgs {
    const float *q;              // [rows][d] queries of this block
    int64_t rows;
    int32_t d, Kp;               // Kp = d rounded up to 16
    const __nv_bfloat16 *tiles;  // [ntiles][2][TCN * Kp] hi, lo in core-matrix layout
    const float *cnorm;          // [nlist]
    int32_t nlist, ntiles, tiles_per_cta;
    float *D;                    // [rows][ldd] squared distances out
    int64_t ldd;
    uint32_t *err;
};

__global__ void __launch_bounds__(TCQ, 1) k_coarse_tc(const CoarseTcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int Kp = a.Kp;
    __nv_bfloat16 *Ahi = reinterpret_cast<__nv_bfloat16 *>(sm);
    __nv_bfloat16 *Alo = Ahi + TCQ * Kp;
    __nv_bfloat16 *Bt = Alo + TCQ * Kp;  // hi then lo, 2 * TCN * Kp
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * TCQ;

    // A: this CTA's queries as bf16 hi/lo; |q|^2 of the thread's own row
    for (int e = tid; e < TCQ * Kp; e += TCQ) {
        const int r = e / Kp, k = e - r * Kp;
        const float x = (r0 + r < a.rows && k < a.d) ? a.q[(r0 + r) * a.d + k] : 0.f;
        __nv_bfloat16 h, l;
        tc::split_bf16(x, h, l);
        const uint32_t o = tc::core_offset(r, k, Kp) >> 1;
        Ahi[o] = h;
        Alo[o] = l;
    }
    float qn = 0.f;
    if (r0 + tid < a.rows)
        for (int k = 0; k < a.d; ++k) {
            const float x = a.q[(r0 + tid) * a.d + k];
            qn = fmaf(x, x, qn);
        }
    if (warp == 0) tc::tmem_alloc(&tmem_base, TCN);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = tmem_base;
    const uint32_t idesc = tc::idesc_bf16_f32(TCQ, TCN);
    const uint32_t sbo = (uint32_t)(Kp / 8) * 128u;
    uint32_t parity = 0;
    bool failed = false;

    const int t0 = blockIdx.y * a.tiles_per_cta;
    const int t1 = min(a.ntiles, t0 + a.tiles_per_cta);
    for (int t = t0; t < t1; ++t) {
        // B: centroid tile t (hi, lo), already in core-matrix layout
        const uint4 *src = reinterpret_cast<const uint4 *>(a.tiles + (size_t)t * 2 * TCN * Kp);
        uint4 *dst = reinterpret_cast<uint4 *>(Bt);
        const int n16 = 2 * TCN * Kp * 2 / 16;
        for (int i = tid; i < n16; i += TCQ) dst[i] = __ldg(src + i);
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
            const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo);
            const uint32_t bh = tc::smem_u32(Bt), bl = bh + TCN * Kp * 2;
            for (int ks = 0; ks < Kp / 16; ++ks) {
                const uint32_t off = 256u * ks;
                const uint64_t dah = tc::smem_desc(ah + off, 128, sbo);
                const uint64_t dal = tc::smem_desc(al + off, 128, sbo);
                const uint64_t dbh = tc::smem_desc(bh + off, 128, sbo);
                const uint64_t dbl = tc::smem_desc(bl + off, 128, sbo);
                tc::mma_bf16(tbase, dah, dbh, idesc, ks > 0 ? 1u : 0u);
                tc::mma_bf16(tbase, dah, dbl, idesc, 1u);
                tc::mma_bf16(tbase, dal, dbh, idesc, 1u);
            }
            tc::mma_commit(&mbar);
        }
        const bool ok = tc::mbar_wait(&mbar, parity, WAIT_LIMIT);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        parity ^= 1u;
        tc::fence_after();
        // epilogue: this thread's row, 256 columns in 8 loads of 32
        const int64_t row = r0 + tid;
        const uint32_t lane_addr = tbase + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < TCN; c0 += 32) {
            float v[32];
            tc::tmem_ld32(lane_addr + c0, v);
            const int l0 = t * TCN + c0;
            if (row < a.rows) {
                float *out = a.D + row * a.ldd + l0;
                if (l0 + 32 <= a.nlist) {
#pragma unroll
                    for (int i = 0; i < 32; i += 4) {
                        float4 o;
                        o.x = qn - 2.f * v[i + 0] + __ldg(a.cnorm + l0 + i + 0);
                        o.y = qn - 2.f * v[i + 1] + __ldg(a.cnorm + l0 + i + 1);
                        o.z = qn - 2.f * v[i + 2] + __ldg(a.cnorm + l0 + i + 2);
                        o.w = qn - 2.f * v[i + 3] + __ldg(a.cnorm + l0 + i + 3);
                        if (((a.ldd | l0) & 3) == 0)
                            *reinterpret_cast<float4 *>(out + i) = o;
                        else {
                            out[i] = o.x;
                            out[i + 1] = o.y;
                            out[i + 2] = o.z;
                            out[i + 3] = o.w;
                        }
                    }
                } else {
                    for (int i = 0; i < 32 && l0 + i < a.nlist; ++i)
                        out[i] = qn - 2.f * v[i] + __ldg(a.cnorm + l0 + i);
                }
            }
        }
        tc::fence_before();
        __syncthreads();
    }
    if (failed) {
        if (tid == 0) atomicOr(a.err, DEV_ERR_TIMEOUT);
        // let an MMA still in flight finish before the tensor memory is freed
        tc::mbar_wait(&mbar, parity, WAIT_LIMIT);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_free(tbase, TCN);
}

// Centroids as TC tiles: [ntiles][hi, lo][TCN rows x Kp] in core-matrix layout,
// rows past nlist zero. Host-side preparation at index upload.
void prepare_centroid_tiles(const float *cent, int32_t nlist, int32_t d, std::vector<uint16_t> &out,
                            int32_t &Kp, int32_t &ntiles) {
    Kp = (d + 15) / 16 * 16;
    ntiles = (nlist + TCN - 1) / TCN;
    out.assign((size_t)ntiles * 2 * TCN * Kp, 0);
    for (int l = 0; l < nlist; ++l) {
        const int t = l / TCN, r = l % TCN;
        uint16_t *hi = out.data() + (size_t)t * 2 * TCN * Kp;
        uint16_t *lo = hi + (size_t)TCN * Kp;
        for (int k = 0; k < d; ++k) {
            const float x = cent[(size_t)l * d + k];
            const uint16_t h = tc::host_bf16_bits(x);
            const uint32_t o = tc::core_offset(r, k, Kp) >> 1;
            hi[o] = h;
            lo[o] = tc::host_bf16_bits(x - tc::host_bf16_float(h));
        }
    }
}

// Distances of `rows` queries to every centroid into D[rows][ldd].
void launch_coarse_tc_dist(const DeviceIndex &ix, const float *q, int64_t rows, float *D,
                           int64_t ldd, uint32_t *err, cudaStream_t st) {
    FA_REQUIRE(ix.centroids_bf16 != nullptr, FA_ERR_ARG, "tensor-core centroid tiles missing");
    CoarseTcArgs a{};
    a.q = q;
    a.rows = rows;
    a.d = ix.d;
    a.Kp = ix.tc_kp;
    a.tiles = reinterpret_cast<const __nv_bfloat16 *>(ix.centroids_bf16);
    a.cnorm = ix.cnorm;
    a.nlist = ix.nlist;
    a.ntiles = ix.tc_ntiles;
    a.D = D;
    a.ldd = ldd;
    a.err = err;
    const int qtiles = (int)((rows + TCQ - 1) / TCQ);
    // enough CTAs for a few waves over the SMs, each reusing its query tile
    int ysplit = std::max(1, std::min(a.ntiles, (num_sms(0) * 4 + qtiles - 1) / qtiles));
    a.tiles_per_cta = (a.ntiles + ysplit - 1) / ysplit;
    ysplit = (a.ntiles + a.tiles_per_cta - 1) / a.tiles_per_cta;
    // at least 116 KB so that no more than one CTA (256 TMEM columns) and at most
    // two share an SM: TMEM allocation never has to wait
    const int smem = std::max((2 * TCQ * a.Kp + 2 * TCN * a.Kp) * 2, 116 * 1024);
    FA_REQUIRE(smem <= 220 * 1024, FA_ERR_ARG, "tensor-core coarse probe supports d <= 128");
    FA_CHECK_CUDA(cudaFuncSetAttribute(k_coarse_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_coarse_tc<<<dim3(qtiles, ysplit), TCQ, smem, st>>>(a);
    FA_CHECK_CUDA(cudaGetLastError());
}

}  // namespace fa
