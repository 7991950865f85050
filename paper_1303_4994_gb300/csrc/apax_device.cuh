// apax_device.cuh -- device building blocks of the APAX codec kernels (sm_103a).
//
// Mapping: one warp owns one codec block.  A block is walked in chunks of
// 256 samples; lane l holds samples 8l..8l+7 of the chunk, i.e. the two
// BFPE groups 2l and 2l+1 (Sec. 6: one exponent per group of 4 samples).
// Everything here is integer arithmetic on IEEE bit patterns, so results are
// bit-identical to any exact implementation of the same reading.
#pragma once

#include <stdint.h>
#include <cuda_runtime.h>

namespace apax {

constexpr int kChunk = 256;  // samples per warp pass
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

// Spread the 32 bits of x to the even bit positions of a 64-bit word.
__device__ __forceinline__ uint64_t spread_even(uint32_t x)
{
    uint64_t v = x;
    v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
    v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
    v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}

// 64-bit position mask of a chunk from two per-lane predicates (group 2l, 2l+1).
__device__ __forceinline__ uint64_t ballot64(bool even_pred, bool odd_pred)
{
    uint32_t be = __ballot_sync(kFull, even_pred), bo = __ballot_sync(kFull, odd_pred);
    return spread_even(be) | (spread_even(bo) << 1);
}

// ---------------------------------------------------------------- integers
__device__ __forceinline__ int32_t sext_w(uint32_t v, int W)
{
    return W >= 32 ? (int32_t)v : ((int32_t)(v << (32 - W)) >> (32 - W));
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

// bits() of a group (Sec. 6 BFPE exponent): max over the values of the
// two's-complement width, 0 for an all-zero group, 31 promoted to 32.
__device__ __forceinline__ int group_exp(int32_t a, int32_t b, int32_t c, int32_t d)
{
    uint32_t mag = (uint32_t)(a ^ (a >> 31)) | (uint32_t)(b ^ (b >> 31)) |
                   (uint32_t)(c ^ (c >> 31)) | (uint32_t)(d ^ (d >> 31));
    uint32_t any = (uint32_t)(a | b | c | d);
    int e = any ? 33 - __clz(mag) : 0;
    return e == 31 ? 32 : e;
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

// ---------------------------------------------------------------- streams
// Redundancy remover (Sec. 5, Sec. 6): S0 the data, S1 first differences,
// S2 second differences (u_1 = q_1 - q_0), all within the block, mod 2^W.
struct Prev2 {  // last two quantised values before this lane's first sample
    int32_t p1, p2;
};

template <int W>
__device__ __forceinline__ void derive(const int32_t (&q)[8], int s, int32_t p1, int32_t p2,
                                       bool block_start, int32_t (&u)[8])
{
    if (s == 0) {
#pragma unroll
        for (int t = 0; t < 8; ++t) u[t] = sext_w((uint32_t)q[t], W);
    } else if (s == 1) {
        uint32_t prev = block_start ? 0u : (uint32_t)p1;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            u[t] = sext_w((uint32_t)q[t] - prev, W);
            prev = (uint32_t)q[t];
        }
    } else {
        uint32_t a = block_start ? 0u : (uint32_t)p2, b = block_start ? 0u : (uint32_t)p1;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            uint32_t v = (uint32_t)q[t] - 2u * b + a;
            if (t == 1 && block_start) v = (uint32_t)q[1] - (uint32_t)q[0];
            u[t] = sext_w(v, W);
            a = b;
            b = (uint32_t)q[t];
        }
    }
}

// ---------------------------------------------------------------- JEE masks
// Greedy JEE pairing (Sec. 6): in every maximal run of diffs in [-1,1] the
// tokens start at even offsets from the run start (a joint token when the
// next diff is also in the run, else a single token).  For a 64-bit mask S of
// such positions, return the even-offset positions.  If `odd_start0`, the run
// that begins at bit 0 continues a run of the previous chunk with its bit 0
// at an odd offset.  Adding a run's start bit to S carries through the run
// and clears it, which separates runs by the parity of their start.
__device__ __forceinline__ uint64_t jee_even_offsets(uint64_t S, bool odd_start0)
{
    const uint64_t EV = 0x5555555555555555ull, OD = ~EV;
    uint64_t R = S & ~(S << 1);
    uint64_t Re = R & EV;
    if (odd_start0) Re &= ~1ull;
    uint64_t X = S + Re;
    // a continued run's start bit was not added, so it stays in runs_odd
    uint64_t runs_even = S & ~X, runs_odd = S & X;
    return (runs_even & EV) | (runs_odd & OD);
}

// Token statistics of one chunk of exponents.
struct ChunkTok {
    int nib;       // nibbles of the tokens that start in this chunk
    bool carry;    // last valid position: small diff at even offset
    int last_e;    // exponent of the last valid group
};

// e0/e1: exponents of groups 2l and 2l+1 of this chunk; G_c: valid groups in
// the chunk; first: this is chunk 0 (its group 0 is the absolute token);
// eprev / carry_in: exponent of the last group of the previous chunk and its
// pairing state.
__device__ __forceinline__ ChunkTok chunk_tokens(int e0, int e1, int G_c, bool first, int eprev,
                                                 bool carry_in)
{
    const unsigned l = lane_id();
    int ep = __shfl_up_sync(kFull, e1, 1);
    if (l == 0) ep = eprev;
    int g0 = 2 * (int)l, g1 = g0 + 1;
    bool v0 = g0 < G_c, v1 = g1 < G_c;
    bool pos0 = !(first && l == 0);  // group 0 of the block has no diff
    int d0 = e0 - ep, d1 = e1 - e0;
    bool s0 = v0 && pos0 && d0 >= -1 && d0 <= 1;
    bool s1 = v1 && d1 >= -1 && d1 <= 1;
    uint64_t S = ballot64(s0, s1);
    uint64_t E = jee_even_offsets(S, carry_in && !first);
    // non-small diffs: one nibble if |d| == 2, else an absolute token (2)
    bool n0 = v0 && pos0 && !s0, n1 = v1 && !s1;
    bool a0 = n0 && (d0 > 2 || d0 < -2), a1 = n1 && (d1 > 2 || d1 < -2);
    uint32_t bn0 = __ballot_sync(kFull, n0), bn1 = __ballot_sync(kFull, n1);
    uint32_t ba0 = __ballot_sync(kFull, a0), ba1 = __ballot_sync(kFull, a1);
    ChunkTok r;
    r.nib = __popcll(E & S) + __popc(bn0) + __popc(bn1) + __popc(ba0) + __popc(ba1) +
            (first ? 2 : 0);
    int lastg = G_c - 1;
    r.carry = (lastg >= 0) && ((E & S) >> lastg & 1);
    r.last_e = __shfl_sync(kFull, (lastg & 1) ? e1 : e0, lastg >> 1);
    return r;
}

}  // namespace apax
