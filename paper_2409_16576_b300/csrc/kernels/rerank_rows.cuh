// Exact squared L2 distances of raw rows against a query, one warp for 32
// rows at a time: shared by the re-rank kernel (step 8) and the scan kernel
// that fuses its exhaustive form.
#pragma once

#include <type_traits>

#include "../fa_internal.h"
#include "warp_topk.cuh"

namespace fa {

// Exact squared L2 of the 32 rows ids[0..31] (one per lane, id < 0 = none)
// against the query in shared memory; lane j returns row j's distance.
// Eight lanes share a row and read consecutive 16-byte pieces of it (4-byte
// words when a row is not a multiple of 16 bytes), so one load instruction
// covers four rows with a full 128-byte request each (d = 128 uint8). The
// loads of all 32 rows are issued before any is summed; the eight partial
// sums of a row are added with three shuffles.
// IP: the negated inner product -<q, x> instead of the squared L2.
// CG: rows written earlier by the same kernel (a page buffer): loads through
// L2 only, never the non-coherent read-only path.
template <typename C, bool CG>
__device__ __forceinline__ C row_piece(const C *p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

template <typename T, typename C, bool IP = false, bool CG = false>
__device__ __forceinline__ float exact_rows(const T *__restrict__ raw, int32_t d,
                                            const float *qs, int64_t my_id) {
    constexpr int EPC = (int)(sizeof(C) / sizeof(T));  // elements per piece
    constexpr int WPC = (int)(sizeof(C) / 4);          // 32-bit words per piece
    constexpr int EPW = EPC / WPC;                     // elements per word
    const int lane = threadIdx.x & 31, r = lane >> 3, c = lane & 7;
    const int pieces = d / EPC;  // per row
    float tot[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) tot[s] = 0.f;
    for (int p0 = 0; p0 < pieces; p0 += 8) {
        const int pc = p0 + c;
        C x[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const long long id = __shfl_sync(FULL, (long long)my_id, 4 * s + r);
            if (id >= 0 && pc < pieces)
                x[s] = row_piece<C, CG>(reinterpret_cast<const C *>(raw + id * (int64_t)d) + pc);
            else
                x[s] = C{};
        }
        if (pc >= pieces) continue;
#pragma unroll
        for (int wd = 0; wd < WPC; ++wd) {
            float qv[EPW];
#pragma unroll
            for (int e = 0; e < EPW; ++e) qv[e] = qs[pc * EPC + wd * EPW + e];
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const uint32_t w = reinterpret_cast<const uint32_t *>(&x[s])[wd];
                float acc = tot[s];
#pragma unroll
                for (int e = 0; e < EPW; ++e) {
                    // a byte b placed in the low mantissa bits of 2^23 reads
                    // as 2^23 + b: one exact subtraction gives b as a float;
                    // an int8 byte flipped in its top bit is b + 128
                    float xv;
                    if constexpr (std::is_same<T, int8_t>::value)
                        xv = __uint_as_float(__byte_perm(w ^ 0x80808080u, 0x4b000000u, 0x7640u + e)) -
                             8388736.0f;
                    else if constexpr (sizeof(T) == 1)
                        xv = __uint_as_float(__byte_perm(w, 0x4b000000u, 0x7640u + e)) - 8388608.0f;
                    else
                        xv = __uint_as_float(w);
                    if (IP) {
                        acc = fmaf(qv[e], xv, acc);
                    } else {
                        const float t = qv[e] - xv;
                        acc = fmaf(t, t, acc);
                    }
                }
                tot[s] = acc;
            }
        }
    }
    float out = 0.f;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        float v = tot[s];
        v += __shfl_xor_sync(FULL, v, 1);
        v += __shfl_xor_sync(FULL, v, 2);
        v += __shfl_xor_sync(FULL, v, 4);
        // row 4s + r' sits on lanes 8r' .. 8r' + 7
        const float mine = __shfl_sync(FULL, v, 8 * (lane & 3));
        if ((lane >> 2) == s) out = mine;
    }
    return IP ? -out : out;
}

// The same for uint8 rows when the query is integral with every coordinate in
// 0..255 (its bytes packed in qp): |x - q| per byte is exact in 8 bits
// (__vabsdiffu4), and a four-byte dot product of it with itself (dp4a) adds
// four squared differences per instruction. Every partial sum is an integer
// below 2^24 for d <= 258, so the float returned equals the FP32 sum of
// squared differences exactly, whatever the order of the additions. Row ids
// travel between lanes as 32 bits (ids below 2^32 - 1); the eight partial
// sums of the 32 rows are added by a three-stage transposing reduction (each
// stage halves the sums a lane holds), 7 shuffles instead of 32.
template <typename C, bool CG = false>
__device__ __forceinline__ float exact_rows_u8int(const uint8_t *__restrict__ raw, int32_t d,
                                                  const uint32_t *qp, int64_t my_id) {
    constexpr int WPC = (int)(sizeof(C) / 4);  // 32-bit words per piece
    const int lane = threadIdx.x & 31, r = lane >> 3, c = lane & 7;
    const int pieces = d / (4 * WPC);
    const uint32_t id32 = my_id < 0 ? 0xffffffffu : (uint32_t)my_id;
    unsigned dd[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) dd[s] = 0u;
    for (int p0 = 0; p0 < pieces; p0 += 8) {
        const int pc = p0 + c;
        C x[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const uint32_t id = __shfl_sync(FULL, id32, 4 * s + r);
            if (id != 0xffffffffu && pc < pieces)
                x[s] = row_piece<C, CG>(reinterpret_cast<const C *>(raw + (size_t)id * (uint32_t)d) + pc);
            else
                x[s] = C{};
        }
        if (pc >= pieces) continue;
#pragma unroll
        for (int wd = 0; wd < WPC; ++wd) {
            const uint32_t qw = qp[pc * WPC + wd];
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const uint32_t w = reinterpret_cast<const uint32_t *>(&x[s])[wd];
                const unsigned ad = __vabsdiffu4(w, qw);  // |x - q| per byte, exact
                dd[s] = __dp4a(ad, ad, dd[s]);
            }
        }
    }
    // dd[s] on lane (r, c) is a partial sum of row 4s + r. Stage h (lane bit
    // b = 4, 2, 1 of c) keeps the half of the sums whose s has bit b equal to
    // the lane's and sends the other half to lane ^ b; after the three stages
    // lane (r, c) holds the whole sum of row 4c + r.
    unsigned e4[4], e2[2];
    const bool b4 = (c & 4) != 0, b2 = (c & 2) != 0, b1 = (c & 1) != 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        e4[j] = (b4 ? dd[j + 4] : dd[j]) + __shfl_xor_sync(FULL, b4 ? dd[j] : dd[j + 4], 4);
#pragma unroll
    for (int j = 0; j < 2; ++j)
        e2[j] = (b2 ? e4[j + 2] : e4[j]) + __shfl_xor_sync(FULL, b2 ? e4[j] : e4[j + 2], 2);
    const unsigned tot = (b1 ? e2[1] : e2[0]) + __shfl_xor_sync(FULL, b1 ? e2[0] : e2[1], 1);
    // row `lane` = 4 (lane >> 2) + (lane & 3) sits on lane 8 (lane & 3) + (lane >> 2)
    return (float)(int)__shfl_sync(FULL, tot, 8 * (lane & 3) + (lane >> 2));
}

// The same for rows a multiple of 32 bytes long, read in 32-byte pieces
// (one 256-bit load each): four lanes share a row, one load instruction
// covers eight rows, and the partial sums take a two-stage transposing
// reduction. Half the loads, id shuffles and address computations of the
// 16-byte form per row, and the same exact integer result. Plain (coherent)
// loads: the rows may sit in mapped host memory.
__device__ __forceinline__ float exact_rows_u8int32(const uint8_t *__restrict__ raw, int32_t d,
                                                    const uint32_t *qp, int64_t my_id) {
    const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    const int pieces = d / 32;
    const uint32_t id32 = my_id < 0 ? 0xffffffffu : (uint32_t)my_id;
    unsigned dd[4] = {0u, 0u, 0u, 0u};
    for (int p0 = 0; p0 < pieces; p0 += 4) {
        const int pc = p0 + c;
        uint32_t x[4][8];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const uint32_t id = __shfl_sync(FULL, id32, 8 * s + g);
            if (id != 0xffffffffu && pc < pieces) {
                const uint8_t *p = raw + (size_t)id * (uint32_t)d + 32 * pc;
                asm("ld.global.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                    : "=r"(x[s][0]), "=r"(x[s][1]), "=r"(x[s][2]), "=r"(x[s][3]), "=r"(x[s][4]),
                      "=r"(x[s][5]), "=r"(x[s][6]), "=r"(x[s][7])
                    : "l"(p));
            } else {
#pragma unroll
                for (int wd = 0; wd < 8; ++wd) x[s][wd] = 0u;
            }
        }
        if (pc >= pieces) continue;
#pragma unroll
        for (int wd = 0; wd < 8; ++wd) {
            const uint32_t qw = qp[pc * 8 + wd];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const unsigned ad = __vabsdiffu4(x[s][wd], qw);
                dd[s] = __dp4a(ad, ad, dd[s]);
            }
        }
    }
    // dd[s] on lane (g, c) is a partial sum of row 8s + g; after the stages
    // on lane bits 2 and 1 lane (g, c) holds the whole sum of row 8c + g
    const bool b2 = (c & 2) != 0, b1 = (c & 1) != 0;
    unsigned e2[2];
#pragma unroll
    for (int j = 0; j < 2; ++j)
        e2[j] = (b2 ? dd[j + 2] : dd[j]) + __shfl_xor_sync(FULL, b2 ? dd[j] : dd[j + 2], 2);
    const unsigned tot = (b1 ? e2[1] : e2[0]) + __shfl_xor_sync(FULL, b1 ? e2[0] : e2[1], 1);
    // row `lane` = 8 (lane >> 3) + (lane & 7) sits on lane 4 (lane & 7) + (lane >> 3)
    return (float)(int)__shfl_sync(FULL, tot, 4 * (lane & 7) + (lane >> 3));
}

// Row pieces: 16 bytes when every row is a multiple of 16 bytes long, else
// 4-byte words.
template <typename T, bool CG = false>
__device__ __forceinline__ float exact_rows_any(const T *__restrict__ raw, int32_t d,
                                                const float *qs, const uint32_t *qp,
                                                bool qint, int64_t my_id, bool ip = false) {
    if constexpr (std::is_same<T, uint8_t>::value) {
        if (qint && !ip) {  // qint needs d % 16 == 0
            if (!CG && d % 32 == 0) return exact_rows_u8int32(raw, d, qp, my_id);
            return exact_rows_u8int<uint4, CG>(raw, d, qp, my_id);
        }
    }
    if ((d * (int)sizeof(T)) % 16 == 0)
        return ip ? exact_rows<T, uint4, true, CG>(raw, d, qs, my_id) : exact_rows<T, uint4, false, CG>(raw, d, qs, my_id);
    return ip ? exact_rows<T, uint32_t, true, CG>(raw, d, qs, my_id)
              : exact_rows<T, uint32_t, false, CG>(raw, d, qs, my_id);
}

// Packs an integral query with every coordinate in 0..255 (the uint8 rows'
// integer form) from its floats qs[0, d) into qp[0, d/4) and returns whether
// it qualifies. One warp; d % 16 == 0 and d <= 258.
__device__ __forceinline__ bool pack_u8_query(const float *qs, int32_t d, uint32_t *qp) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    for (int j4 = lane; j4 < d / 4; j4 += 32) {
        uint32_t wq = 0;
        for (int e = 0; e < 4; ++e) {
            const float v = qs[4 * j4 + e];
            ok = ok && v >= 0.f && v <= 255.f && v == rintf(v);
            wq |= (ok ? (uint32_t)v : 0u) << (8 * e);
        }
        qp[j4] = wq;
    }
    const bool all = __all_sync(FULL, ok);
    __syncwarp();
    return all;
}

}  // namespace fa
