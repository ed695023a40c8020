// Warp-level selection of the n smallest (distance, id) pairs (step 7 of the
// filtering path: the GPU "sorts all distances and returns the top-n").
//
// A pair is packed into one 64-bit key: the high word is the distance mapped
// to an unsigned integer that orders like the float, the low word the id. Key
// order is therefore (distance asc, id asc), which makes every selection
// deterministic. Selection is a bitonic network held in registers: element e
// of a warp-wide array of 32*R keys sits in register e / 32 of lane e % 32.
#pragma once
#include <stdint.h>

namespace fa {

constexpr uint64_t KEY_INF = ~0ull;
constexpr uint32_t FULL = 0xffffffffu;

__device__ __forceinline__ uint32_t f2o(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float o2f(uint32_t o) {
    uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    return __uint_as_float(u);
}

__device__ __forceinline__ uint64_t make_key(float d, uint32_t id) {
    return ((uint64_t)f2o(d) << 32) | id;
}

__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int m) {
    uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
    lo = __shfl_xor_sync(FULL, lo, m);
    hi = __shfl_xor_sync(FULL, hi, m);
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
    uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
    lo = __shfl_sync(FULL, lo, src);
    hi = __shfl_sync(FULL, hi, src);
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a < b ? b : a; }

// One bitonic stage over 32*R keys: compare element e with e ^ STRIDE,
// ascending where (e & SIZE) == 0. SIZE and STRIDE are compile-time constants
// so that every register index below is static (no local memory).
template <int R, int SIZE, int STRIDE>
__device__ __forceinline__ void bitonic_stage(uint64_t (&v)[R]) {
    const int lane = threadIdx.x & 31;
    if constexpr (STRIDE >= 32) {
        constexpr int RS = STRIDE >> 5;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if ((r & RS) == 0) {
                const bool up = (((r << 5) & SIZE) == 0);
                const uint64_t a = v[r], b = v[r | RS];
                const uint64_t lo = umin64(a, b), hi = umax64(a, b);
                v[r] = up ? lo : hi;
                v[r | RS] = up ? hi : lo;
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = (r << 5) | lane;
            const bool up = ((e & SIZE) == 0);
            const uint64_t o = shfl_xor64(v[r], STRIDE);
            const bool lower = (lane & STRIDE) == 0;
            v[r] = (lower == up) ? umin64(v[r], o) : umax64(v[r], o);
        }
    }
}

template <int R, int SIZE, int STRIDE>
__device__ __forceinline__ void bitonic_stages_from(uint64_t (&v)[R]) {
    bitonic_stage<R, SIZE, STRIDE>(v);
    if constexpr (STRIDE > 1) bitonic_stages_from<R, SIZE, STRIDE / 2>(v);
}

template <int R, int SIZE>
__device__ __forceinline__ void bitonic_sort_from(uint64_t (&v)[R]) {
    bitonic_stages_from<R, SIZE, SIZE / 2>(v);
    if constexpr (SIZE < 32 * R) bitonic_sort_from<R, SIZE * 2>(v);
}

// Sorts 32*R keys ascending.
template <int R>
__device__ __forceinline__ void bitonic_sort(uint64_t (&v)[R]) {
    bitonic_sort_from<R, 2>(v);
}

// Sorts a bitonic sequence of 32*R keys ascending.
template <int R>
__device__ __forceinline__ void bitonic_merge(uint64_t (&v)[R]) {
    bitonic_stages_from<R, 64 * R, 16 * R>(v);
}

// L (sorted, 32*R keys) <- the 32*R smallest of L and B (sorted, 32*R keys).
// min(L[i], B[32R-1-i]) is bitonic and holds exactly those keys.
template <int R>
__device__ __forceinline__ void merge_sorted(uint64_t (&L)[R], const uint64_t (&B)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) L[r] = umin64(L[r], shfl_xor64(B[R - 1 - r], 31));
    bitonic_merge<R>(L);
}

// L (sorted, 32*R) <- smallest 32*R of L and 32 sorted keys b (one per lane).
template <int R>
__device__ __forceinline__ void merge_sorted32(uint64_t (&L)[R], uint64_t b) {
    L[R - 1] = umin64(L[R - 1], shfl_xor64(b, 31));
    bitonic_merge<R>(L);
}

// The 32 smallest of a sorted warp-wide list of 32 keys (one per lane) and
// the keys b of the lanes in mask (each below the list's last key and
// distinct from its keys), inserted one at a time: the result equals
// sorting b and merging it with merge_sorted32, at about a tenth of the
// instructions when few lanes are set.
__device__ __forceinline__ void insert_sorted32(uint64_t &L, uint64_t b, uint32_t mask) {
    const int lane = threadIdx.x & 31;
    while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1u;
        const uint64_t x = shfl64(b, src);
        const int pos = __popc(__ballot_sync(FULL, L < x));
        uint32_t lo = (uint32_t)L, hi = (uint32_t)(L >> 32);
        lo = __shfl_up_sync(FULL, lo, 1);
        hi = __shfl_up_sync(FULL, hi, 1);
        const uint64_t up = ((uint64_t)hi << 32) | lo;
        L = lane < pos ? L : (lane == pos ? x : up);
    }
}

// Element e of a warp-wide array (same value on every lane).
// (a mask blend rather than a select on e / 32, which the compiler may turn
// into an indexed array in local memory)
template <int R>
__device__ __forceinline__ uint64_t warp_elem(const uint64_t (&v)[R], int e) {
    uint64_t t = 0;
    const int re = e >> 5;
#pragma unroll
    for (int r = 0; r < R; ++r) t |= v[r] & (0ull - (uint64_t)(re == r));
    return shfl64(t, e & 31);
}

// Running top-n of a stream of keys for one warp. The sorted list lives in
// registers; keys below the current n-th best are appended to a 64-entry
// shared-memory buffer and merged in blocks of 32.
template <int R>
struct WarpTopK {
    uint64_t L[R];
    uint64_t thr;   // current n-th smallest key (KEY_INF until n keys are held)
    uint64_t *buf;  // 64 keys in shared memory, private to the warp
    int cnt;        // keys in buf (warp-uniform)
    int n;          // keys wanted, 1 <= n <= 32*R
    unsigned long long *sthr;  // optional threshold shared by the CTA's warps
    // Optional, with sthr: one slot per warp of the CTA (nslots of them, all
    // KEY_INF at the start of a query). Warp w publishes its t-th smallest key,
    // t = ceil(n / nslots). The nslots warps then hold at least n distinct keys
    // at or below the largest published key, so that key bounds the CTA's
    // n-th smallest: a much tighter threshold than any one warp's n-th.
    unsigned long long *slots;
    int nslots, slot;

    __device__ __forceinline__ void init(uint64_t *wbuf, int n_) {
        sthr = nullptr;
        slots = nullptr;
        nslots = 0;
        slot = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) L[r] = KEY_INF;
        thr = KEY_INF;
        buf = wbuf;
        cnt = 0;
        n = n_;
    }

    __device__ __forceinline__ void merge32() {
        const int lane = threadIdx.x & 31;
        __syncwarp();
        uint64_t b = lane < cnt ? buf[lane] : KEY_INF;
        uint64_t bb[1] = {b};
        bitonic_sort<1>(bb);
        merge_sorted32<R>(L, bb[0]);
        thr = warp_elem<R>(L, n - 1);
        // any warp's n-th best bounds the CTA's n-th best from above
        if (sthr && thr != KEY_INF && (threadIdx.x & 31) == 0) atomicMin(sthr, (unsigned long long)thr);
        if (slots) {
            const uint64_t mine = warp_elem<R>(L, (n + nslots - 1) / nslots - 1);
            if (lane == 0) *(volatile unsigned long long *)(slots + slot) = mine;
            __syncwarp();
            uint64_t hi = lane < nslots ? *(volatile unsigned long long *)(slots + lane) : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) hi = umax64(hi, shfl_xor64(hi, o));
            if (hi != KEY_INF && lane == 0) atomicMin(sthr, (unsigned long long)hi);
        }
        int rem = cnt - 32;
        uint64_t x = (rem > 0 && lane < rem) ? buf[32 + lane] : 0;
        __syncwarp();
        if (rem > 0 && lane < rem) buf[lane] = x;
        cnt = rem > 0 ? rem : 0;
        __syncwarp();
    }

    // Offers one key per lane (pass = false lanes offer nothing).
    __device__ __forceinline__ void push(uint64_t key, bool valid) {
        const int lane = threadIdx.x & 31;
        uint64_t t = thr;
        if (sthr) t = umin64(t, *(volatile unsigned long long *)sthr);
        const bool pass = valid && key < t;
        const uint32_t m = __ballot_sync(FULL, pass);
        if (m) {
            const int pos = cnt + __popc(m & ((1u << lane) - 1u));
            if (pass) buf[pos] = key;
            cnt += __popc(m);
            if (cnt >= 32) merge32();
        }
    }

    __device__ __forceinline__ void finish() {
        if (cnt > 0) merge32();
    }
};

}  // namespace fa
