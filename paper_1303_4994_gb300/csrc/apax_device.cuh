// apax_device.cuh -- device building blocks of the APAX codec kernels (sm_103a).
//
// Element-type traits, the attenuator's quantiser and the decoder's exact
// rounding.  Everything here is integer arithmetic on IEEE bit patterns, so
// results are bit-identical to any exact implementation of the same reading.
#pragma once

#include <stdint.h>
#include <cuda_runtime.h>

namespace apax {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------- dtypes
// W: width of the integer domain the streams live in (mod 2^W).
// Q: float quantiser precision (|q| <= 2^Q).  H: block header bits (Sec. 6:
// 4 bytes for integers, 6 for floats).
template <int DT> struct DT_;
template <> struct DT_<1> { using raw = int8_t;  static constexpr int S = 1, W = 8,  F = 0, Q = 0,  H = 32; };
template <> struct DT_<2> { using raw = int16_t; static constexpr int S = 2, W = 16, F = 0, Q = 0,  H = 32; };
template <> struct DT_<3> { using raw = int32_t; static constexpr int S = 4, W = 32, F = 0, Q = 0,  H = 32; };
template <> struct DT_<4> {
    using raw = float; using bits = uint32_t;
    static constexpr int S = 4, W = 32, F = 1, Q = 23, H = 48, MB = 23, BIAS = 127, EMAX = 255;
    static constexpr int P = 24, EMIN_U = -149, EMAXV = 127;
};
template <> struct DT_<5> {
    using raw = double; using bits = uint64_t;
    static constexpr int S = 8, W = 32, F = 1, Q = 29, H = 48, MB = 52, BIAS = 1023, EMAX = 2047;
    static constexpr int P = 53, EMIN_U = -1074, EMAXV = 1023;
};

// Lane storage of one sample: sign-extended int for integer types, the IEEE
// bit pattern for floats.
template <int DT> struct LaneT { using t = int32_t; };
template <> struct LaneT<4> { using t = uint32_t; };
template <> struct LaneT<5> { using t = uint64_t; };

// ---------------------------------------------------------------- warp ops
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31; }

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    const unsigned l = lane_id();
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T t = __shfl_up_sync(kFull, v, d);
        if (l >= (unsigned)d) v += t;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v)
{
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        uint64_t t = __shfl_xor_sync(kFull, v, d);
        v = t > v ? t : v;
    }
    return v;
}

// ---------------------------------------------------------------- integers
__device__ __forceinline__ int32_t sext_w(uint32_t v, int W)
{
    return W >= 32 ? (int32_t)v : ((int32_t)(v << (32 - W)) >> (32 - W));
}

// Bits [pos, pos + len) of v sign-extended from bit pos + len - 1 (len = 0
// gives 0; pos + len <= 32 here).
__device__ __forceinline__ int32_t bfe_s32(uint32_t v, uint32_t pos, uint32_t len)
{
    int32_t r;
    asm("bfe.s32 %0, %1, %2, %3;" : "=r"(r) : "r"(v), "r"(pos), "r"(len));
    return r;
}

// Round-half-to-even of t / 2^s, s >= 1, |t| < 2^62.
__device__ __forceinline__ int64_t rne_shift_s64(int64_t t, int s)
{
    if (s >= 63) return 0;
    return (t + ((int64_t)1 << (s - 1)) - 1 + ((t >> s) & 1)) >> s;
}

// Round-half-to-even of P / 2^s for P < 2^62; s <= 0 multiplies.
__device__ __forceinline__ uint64_t rne_shift_u64(uint64_t P, int s)
{
    if (s <= 0) return P << (-s);
    if (s >= 64) return 0;
    return (P + ((uint64_t)1 << (s - 1)) - 1 + ((P >> s) & 1)) >> s;
}

// ---------------------------------------------------------------- attenuator
struct Code {
    int k, m;
    bool zero;  // code 4095: the zero attenuator
    __device__ __forceinline__ explicit Code(int c) : k(c >> 7), m(c & 127), zero(c == 4095) {}
};

// Block exponent of a float block from its largest magnitude bit pattern:
// max|x| = f 2^Eb with f in [0.5, 1); 0 for an all-zero block.
template <int DT>
__device__ __forceinline__ int block_exp_from_maxbits(uint64_t mb)
{
    using T = DT_<DT>;
    if (mb == 0) return 0;
    int bexp = (int)(mb >> T::MB);
    if (bexp) return bexp - (T::BIAS - 1);
    int nb = 64 - __clzll(mb);  // subnormal: value = mant 2^(1-BIAS-MB)
    return nb + (1 - T::BIAS - T::MB);
}

// Quantiser (Sec. 6 attenuator): q = RNE(x a(c)) for integers, and
// q = RNE(x 2^(Q-Eb) a(c)) for floats, the exact product rounded once.
template <int DT>
__device__ __forceinline__ int32_t quantise(typename LaneT<DT>::t v, const Code &c, int Eb)
{
    using T = DT_<DT>;
    if (c.zero) return 0;
    if constexpr (!T::F) {
        if constexpr (DT == 3) {
            int64_t t = (int64_t)v * (256 - c.m);
            return (int32_t)rne_shift_s64(t, 8 + c.k);
        } else {
            int32_t t = v * (256 - c.m);
            int s = 8 + c.k;
            if (s >= 25) return 0;  // |t| < 2^23
            return (t + (1 << (s - 1)) - 1 + ((t >> s) & 1)) >> s;
        }
    } else {
        using B = typename T::bits;
        constexpr B mmask = ((B)1 << T::MB) - 1;
        int bexp = (int)((v >> T::MB) & (B)T::EMAX);
        uint64_t M = (uint64_t)(v & mmask) | (bexp ? ((uint64_t)1 << T::MB) : 0);
        int ex = (bexp ? bexp : 1) - T::BIAS - T::MB;
        int sh = (8 + c.k) - (T::Q - Eb + ex);
        uint64_t q = rne_shift_u64(M * (uint64_t)(256 - c.m), sh);
        bool neg = (v >> (sizeof(B) * 8 - 1)) & 1;
        return neg ? -(int32_t)q : (int32_t)q;
    }
}

// Decoder reciprocal table R[m] = RNE(2^32 / (256 - m)), built once per CTA
// with exact integer division.
__device__ __forceinline__ uint32_t recip_entry(int m)
{
    uint64_t d = 256 - m, num = 1ull << 32;
    uint64_t q = num / d, r = num - q * d;
    if (2 * r > d || (2 * r == d && (q & 1))) q += 1;
    return (uint32_t)q;
}

// Round the exact value V 2^e (V != 0) to the float format of DT with ties to
// even, saturating beyond the largest finite value; returns the bit pattern.
template <int DT>
__device__ __forceinline__ typename DT_<DT>::bits round_to_format(int64_t V, int e)
{
    using T = DT_<DT>;
    using B = typename T::bits;
    if (V == 0) return 0;
    bool neg = V < 0;
    uint64_t A = neg ? (uint64_t)(-V) : (uint64_t)V;
    int nb = 64 - __clzll(A);
    int top = e + nb - 1;
    int u = top - (T::P - 1);
    if (u < T::EMIN_U) u = T::EMIN_U;
    uint64_t mant = rne_shift_u64(A, u - e);
    if (mant >> T::P) {  // carry out of the rounding
        mant >>= 1;
        u += 1;
    }
    B out;
    if (mant == 0) {
        out = 0;
    } else if (u + T::P - 1 > T::EMAXV) {
        out = ((B)(T::EMAX - 1) << T::MB) | (((B)1 << T::MB) - 1);  // largest finite
    } else if (!(mant >> (T::P - 1))) {
        out = (B)mant;  // subnormal (u == EMIN_U)
    } else {
        B bexp = (B)(u + T::P - 1 + T::BIAS);
        out = (bexp << T::MB) | ((B)mant & (((B)1 << T::MB) - 1));
    }
    if (neg) out |= (B)1 << (sizeof(B) * 8 - 1);
    return out;
}

}  // namespace apax
