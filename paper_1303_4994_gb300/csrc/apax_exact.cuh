// apax_exact.cuh -- exact integer accumulation and correctly rounded
// conversion to binary64, for the profiler's reconstruction sums (Sec. 4).
//
// A block's sums of x, y, x^2, xy, y^2 and (x-y)^2 are exact integers times
// a power of two.  They are accumulated in 64-, 128- or 256-bit two's
// complement integers, summed across the warp with REDUX on 22-bit chunks
// (exact, order free), and rounded once (ties to even) to binary64.
#pragma once

#include "apax_device.cuh"

namespace apax {

typedef __int128 i128;
typedef unsigned __int128 u128;

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ uint64_t warp_sum_u64_mod(uint64_t v)
{
    uint32_t c0 = (uint32_t)(v & 0x3FFFFFu), c1 = (uint32_t)((v >> 22) & 0x3FFFFFu),
             c2 = (uint32_t)(v >> 44);
    uint64_t s0 = __reduce_add_sync(kFull, c0), s1 = __reduce_add_sync(kFull, c1),
             s2 = __reduce_add_sync(kFull, c2);
    return s0 + (s1 << 22) + (s2 << 44);
}

__device__ __forceinline__ int64_t warp_sum_i64(int64_t v)
{
    return (int64_t)warp_sum_u64_mod((uint64_t)v);
}

__device__ __forceinline__ u128 warp_sum_u128_mod(u128 v)
{
    u128 out = 0;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        uint32_t ch = (uint32_t)(v >> (22 * c)) & 0x3FFFFFu;
        uint32_t s = __reduce_add_sync(kFull, ch);
        out += (u128)s << (22 * c);
    }
    return out;
}

__device__ __forceinline__ i128 warp_sum_i128(i128 v) { return (i128)warp_sum_u128_mod((u128)v); }

// 256-bit two's complement integer, 4 little-endian limbs.
struct W256 {
    uint64_t l[4];
};

__device__ __forceinline__ void w256_zero(W256 &a)
{
#pragma unroll
    for (int i = 0; i < 4; ++i) a.l[i] = 0;
}

// a += (neg ? -1 : 1) * t * 2^p, 0 <= p, t < 2^128, p + bits(t) < 256.
__device__ __forceinline__ void w256_add(W256 &a, u128 t, int p, bool neg)
{
    const uint64_t lo = (uint64_t)t, hi = (uint64_t)(t >> 64);
    const int li = p >> 6, sh = p & 63;
    uint64_t t0 = lo << sh;
    uint64_t t1 = sh ? ((hi << sh) | (lo >> (64 - sh))) : hi;
    uint64_t t2 = sh ? (hi >> (64 - sh)) : 0;
    uint64_t add[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        add[i] = (i == li) ? t0 : (i == li + 1) ? t1 : (i == li + 2) ? t2 : 0;
    if (neg) {  // two's complement negate the 256-bit addend
        uint64_t c = 1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint64_t v = ~add[i] + c;
            c = (c && v == 0) ? 1 : 0;
            add[i] = v;
        }
    }
    uint64_t carry = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint64_t s = a.l[i] + add[i];
        uint64_t c1 = s < a.l[i];
        uint64_t s2 = s + carry;
        uint64_t c2 = s2 < s;
        a.l[i] = s2;
        carry = c1 | c2;
    }
}

__device__ __forceinline__ W256 warp_sum_w256(const W256 &a)
{
    // 12 chunks of 22 bits cover 264 bits; sums < 2^27 per chunk
    W256 r;
    w256_zero(r);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const int b = 22 * c, li = b >> 6, sh = b & 63;
        uint64_t v = a.l[li] >> sh;
        if (sh > 42 && li < 3) v |= a.l[li + 1] << (64 - sh);
        uint32_t ch = (uint32_t)v & 0x3FFFFFu;
        uint32_t s = __reduce_add_sync(kFull, ch);
        w256_add(r, (u128)s, b, false);
    }
    return r;
}

// ---------------------------------------------------------------- rounding
// Correctly rounded binary64 of A 2^e (A > 0 given as up to 256 bits in
// limbs, nb = bit length), ties to even, subnormals, overflow to infinity.
__device__ __forceinline__ double round_limbs(const uint64_t (&L)[4], int nb, int e, bool neg)
{
    if (nb == 0) return neg ? -0.0 : 0.0;
    const int top = e + nb - 1;
    int u = top - 52;
    if (u < -1074) u = -1074;
    const int cut = u - e;  // number of low bits dropped (may be <= 0)
    uint64_t mant;
    bool half = false, sticky = false;
    if (cut <= 0) {
        mant = L[0] << (-cut);  // nb <= 53 here
    } else {
        // mant = bits [cut, nb) ; half = bit cut-1 ; sticky = any below
        auto bit = [&](int i) -> uint64_t { return (L[i >> 6] >> (i & 63)) & 1ull; };
        const int li = cut >> 6, sh = cut & 63;
        mant = L[li] >> sh;
        if (sh && li < 3) mant |= L[li + 1] << (64 - sh);
        const int len = nb - cut;  // <= 53
        if (len < 64) mant &= (len <= 0 ? 0ull : ((1ull << len) - 1));
        if (len <= 0) mant = 0;
        half = bit(cut - 1);
        const int sb = cut - 1;  // bits [0, sb)
        const int sli = sb >> 6, ssh = sb & 63;
        for (int i = 0; i < sli && !sticky; ++i) sticky = L[i] != 0;
        if (!sticky && ssh) sticky = (L[sli] & ((1ull << ssh) - 1)) != 0;
    }
    if (half && (sticky || (mant & 1))) mant += 1;
    if (mant >> 53) {  // carry out of the rounding
        mant >>= 1;
        u += 1;
    }
    uint64_t bits;
    if (mant == 0) {
        bits = 0;
    } else if (!(mant >> 52)) {
        bits = mant;  // subnormal: u == -1074
    } else if (u + 52 > 1023) {
        bits = 0x7ff0000000000000ull;  // overflow rounds to infinity
    } else {
        bits = ((uint64_t)(u + 52 + 1023) << 52) | (mant & 0x000fffffffffffffull);
    }
    if (neg) bits |= 0x8000000000000000ull;
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ int nbits_u64(uint64_t v) { return v ? 64 - __clzll(v) : 0; }

__device__ __forceinline__ double round_u128(u128 A, int e)
{
    uint64_t L[4] = {(uint64_t)A, (uint64_t)(A >> 64), 0, 0};
    int nb = L[1] ? 64 + nbits_u64(L[1]) : nbits_u64(L[0]);
    return round_limbs(L, nb, e, false);
}

__device__ __forceinline__ double round_i128(i128 V, int e)
{
    bool neg = V < 0;
    u128 A = neg ? (u128)(-V) : (u128)V;
    uint64_t L[4] = {(uint64_t)A, (uint64_t)(A >> 64), 0, 0};
    int nb = L[1] ? 64 + nbits_u64(L[1]) : nbits_u64(L[0]);
    return round_limbs(L, nb, e, neg);
}

__device__ __forceinline__ double round_w256(const W256 &a, int e)
{
    bool neg = (a.l[3] >> 63) & 1;
    uint64_t L[4];
    if (neg) {
        uint64_t c = 1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint64_t v = ~a.l[i] + c;
            c = (c && v == 0) ? 1 : 0;
            L[i] = v;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) L[i] = a.l[i];
    }
    int nb = 0;
#pragma unroll
    for (int i = 3; i >= 0; --i)
        if (!nb && L[i]) nb = 64 * i + nbits_u64(L[i]);
    return round_limbs(L, nb, e, neg);
}

// ---------------------------------------------------------------- shared superaccumulator
// Fallback for blocks whose values span too many binades for the 256-bit
// window: int64 digits of 32 bits at positions LO + 32 i, updated with
// shared-memory atomics by all lanes (exact, order free).
template <int ND, int LO>
struct SmemAcc {
    long long *d;  // ND digits in shared memory
    __device__ __forceinline__ void clear()
    {
        for (int i = lane_id(); i < ND; i += 32) d[i] = 0;
        __syncwarp();
    }
    __device__ __forceinline__ void add(u128 v, int e, bool neg)
    {
        if (v == 0) return;
        const int p = e - LO;
        const int di = p >> 5, sh = p & 31;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint64_t chunk = (uint64_t)(v >> (32 * i)) & 0xffffffffull;
            if (!chunk) continue;
            uint64_t t = chunk << sh;
            long long lo = (long long)(t & 0xffffffffull), hi = (long long)(t >> 32);
            if (neg) { lo = -lo; hi = -hi; }
            if (lo) atomicAdd((unsigned long long *)&d[di + i], (unsigned long long)lo);
            if (hi) atomicAdd((unsigned long long *)&d[di + i + 1], (unsigned long long)hi);
        }
    }
    // Round to binary64 in place (one lane, after __syncwarp; destroys the
    // digits).
    __device__ double round_inplace()
    {
        long long carry = 0;
        for (int i = 0; i < ND; ++i) {
            long long t = d[i] + carry;
            long long low = (long long)((unsigned long long)t & 0xffffffffull);
            carry = (t - low) / 4294967296LL;
            d[i] = low;
        }
        const bool neg = carry < 0;
        if (neg) {
            unsigned long long c = 1;
            for (int i = 0; i < ND; ++i) {
                unsigned long long t = (unsigned long long)((uint32_t)~(uint32_t)d[i]) + c;
                d[i] = (long long)(t & 0xffffffffull);
                c = t >> 32;
            }
        }
        int top = -1;
        for (int i = ND - 1; i >= 0; --i)
            if (d[i]) { top = i; break; }
        if (top < 0) return 0.0;
        // the top three digits as one 96-bit value; its leading one becomes
        // bit 63 of a 64-bit window, and everything below folds into a
        // sticky bit (bit 0, below the rounding point)
        const uint32_t w2 = (uint32_t)d[top];
        const uint32_t w1 = top >= 1 ? (uint32_t)d[top - 1] : 0u;
        const uint32_t w0 = top >= 2 ? (uint32_t)d[top - 2] : 0u;
        const u128 V = ((u128)w2 << 64) | ((u128)w1 << 32) | (u128)w0;
        const int sh = 32 - __clz(w2);  // 1..32
        const uint64_t win = (uint64_t)(V >> sh);
        bool st = (V & (((u128)1 << sh) - 1)) != 0;
        for (int i = 0; i < top - 2 && !st; ++i) st = d[i] != 0;
        const int lowbit = 32 * (top - 2) + sh;  // position of the window's bit 0
        uint64_t L[4] = {win | (st ? 1ull : 0ull), 0, 0, 0};
        return round_limbs(L, 64, lowbit + LO, neg);
    }
};

}  // namespace apax
